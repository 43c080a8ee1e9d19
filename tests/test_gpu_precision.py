"""Per-circuit error of the complex64 path against the FP64 oracle, with and
without commutation-aware fusion, on the random layered workload (Haar U(2)
on every qubit + CZ on a seeded perfect matching per layer) at 24 qubits,
depth 40 (1440 gates): fidelity and max amplitude error, asserted under the
rounding bound derived gate by gate in gpu_util. complex128 on the same
circuit meets the oracle to 1e-12."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, c64_circuit_bound, fidelity_loss_bound, host

pytestmark = pytest.mark.gpu

N_QUBITS, DEPTH = 24, 40


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def circuit_and_oracle():
    circ = synth.random_layered(N_QUBITS, DEPTH, seed=0)
    want = oracle.run_circuit(circ, synth.basis_state(N_QUBITS, 0))
    return circ, want


def _run(api, ops, dtype):
    x = torch.zeros(1 << N_QUBITS, dtype=dtype, device="cuda")
    x[0] = 1
    for op in ops:
        api.apply(op, x, x)
    return host(x)


def _ks(circ_gates, ops, fused):
    """Qubit count per applied op for the bound; CZ (entries 0, +-1) counts 0."""
    if not fused:
        return [0 if g.name == "cz" else g.k for g in circ_gates]
    return [op.info()["k"] for op in ops]


@pytest.mark.parametrize("fused", [False, True])
def test_random24_c64_error_vs_oracle(api, circuit_and_oracle, fused):
    circ, want = circuit_and_oracle
    if fused:
        ops = api.build_fused(circ.gates, N_QUBITS, 3, 6, dtype=torch.complex64, commuting=True)
    else:
        ops = [api.build(g, N_QUBITS, dtype=torch.complex64) for g in circ.gates]
    got = _run(api, ops, torch.complex64)
    B = c64_circuit_bound(_ks(circ.gates, ops, fused))
    err = oracle.max_abs_err(got, want)
    loss = 1.0 - oracle.fidelity(got, want)
    print(f"random-{N_QUBITS} d{DEPTH} c64 fused={fused}: ops {len(ops)}, max|d amp| {err:.3e}, "
          f"1-F {loss:.3e}, bound {B:.3e} / {fidelity_loss_bound(B):.3e}")
    assert err <= B
    assert loss <= fidelity_loss_bound(B)
    # the state really moved away from |0...0> and kept its norm
    assert abs(got[0]) < 0.01 and abs(oracle.norm2(got) - 1.0) <= 2 * B


@pytest.mark.parametrize("fused", [False, True])
def test_random24_c128_vs_oracle(api, circuit_and_oracle, fused):
    circ, want = circuit_and_oracle
    if fused:
        ops = api.build_fused(circ.gates, N_QUBITS, 3, 6, dtype=torch.complex128, commuting=True)
    else:
        ops = [api.build(g, N_QUBITS) for g in circ.gates]
    got = _run(api, ops, torch.complex128)
    assert oracle.max_abs_err(got, want) <= TOL_C128
    assert 1.0 - oracle.fidelity(got, want) <= 1e-20 + 1e-13
