"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This package holds input generation only: circuits as plain data (gate lists
with targets, fixed gate matrices, parameter indices and Pauli generators),
random states and Pauli-sum observables. It applies no gate, forms no
Kronecker product, multiplies no diagonals and reduces no state; those are
the method's arithmetic and live, independently, in ``oracle/`` (CPU) and in
the CUDA library (GPU).
"""

from .circuits import (  # noqa: F401
    Gate,
    Circuit,
    Observable,
    H,
    X,
    CNOT,
    CZ,
    SWAP,
    cphase,
    haar_u2,
    ghz,
    qft,
    random_layered,
    ansatz,
    ansatz_observable,
    tfim,
    magnetisation_observable,
    qaoa_instance,
    qaoa_batch,
    random_state,
    basis_state,
    random_gate,
    pauli_masks,
)
