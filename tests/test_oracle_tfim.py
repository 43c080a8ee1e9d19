"""Pins for the oracle on the Trotterised transverse-field Ising workload (the
paper's Hamiltonian-simulation benchmark, Section VII: 1D TFIM by
Trotterisation, read out as the average magnetisation). The facts used here
do not come from the oracle: closed forms of the two decoupled limits, and
the exact propagator exp(-iHt) of the dense Hamiltonian (scipy.linalg.expm
of a matrix assembled with numpy.kron), which a first-order Trotter product
approaches linearly in the step size.
"""

import math

import numpy as np
import pytest

import oracle
import synth

scipy_linalg = pytest.importorskip("scipy.linalg")

_P = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def _dense_string(n, letters):
    """Kronecker product with qubit n-1 first (qubit 0 is the least
    significant index bit)."""
    m = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        m = np.kron(m, _P[letters.get(q, "I")])
    return m


def _dense_tfim(n, J, h):
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for i in range(n - 1):
        H -= J * _dense_string(n, {i: "Z", i + 1: "Z"})
    for i in range(n):
        H -= h * _dense_string(n, {i: "X"})
    return H


def _mz_dense(n, psi):
    M = sum(_dense_string(n, {i: "Z"}) for i in range(n)) / n
    return float(np.vdot(psi, M @ psi).real)


def _run(circ):
    return oracle.run_circuit(circ, synth.basis_state(circ.n, 0))


@pytest.mark.parametrize("steps", [1, 3, 8])
def test_zero_coupling_precession_closed_form(steps):
    """J = 0: the qubits decouple and every one precesses about X, so from
    |0...0> the magnetisation is cos(2 h t) at t = steps * dt, exactly (the
    field gates commute, so Trotterisation makes no error)."""
    n, dt, h = 5, 0.13, 0.9
    c = synth.tfim(n, steps, dt, J=0.0, h=h)
    psi = _run(c)
    m = oracle.expect(psi, synth.magnetisation_observable(n)).real
    assert abs(m - math.cos(2 * h * steps * dt)) < 1e-13
    assert abs(oracle.norm2(psi) - 1.0) < 1e-13


def test_zero_field_is_stationary():
    """h = 0: |0...0> is an eigenstate of every Z_i Z_{i+1}, so the state only
    gains the phase exp(i J t (n-1)) and the magnetisation stays 1."""
    n, steps, dt, J = 6, 4, 0.21, 1.3
    psi = _run(synth.tfim(n, steps, dt, J=J, h=0.0))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = np.exp(1j * J * steps * dt * (n - 1))
    assert np.max(np.abs(psi - want)) < 1e-14
    assert abs(oracle.expect(psi, synth.magnetisation_observable(n)).real - 1.0) < 1e-14


def test_trotter_converges_linearly_to_exact_propagator():
    """First-order Trotter: the state error against exp(-iHT)|0> shrinks
    about twofold when the step halves, and the magnetisation converges to
    that of the exact state. A sign error in J or h, or a wrong angle
    convention, converges to the wrong limit and fails this."""
    n, J, h, T = 6, 1.0, 0.7, 0.6
    H = _dense_tfim(n, J, h)
    e0 = synth.basis_state(n, 0)
    exact = scipy_linalg.expm(-1j * T * H) @ e0
    errs = []
    for steps in (10, 20, 40):
        psi = _run(synth.tfim(n, steps, T / steps, J=J, h=h))
        errs.append(float(np.linalg.norm(psi - exact)))
    assert 1.7 < errs[0] / errs[1] < 2.3
    assert 1.7 < errs[1] / errs[2] < 2.3
    # first-order bound (T^2 / 2m) * sum ||[A_i, B_j]||: bond i fails to
    # commute with the fields on its two ends, each commutator of norm 2 J h
    bound = T * T / (2 * 40) * 2 * (n - 1) * 2 * J * h
    assert errs[2] < bound
    m = oracle.expect(_run(synth.tfim(n, 400, T / 400, J=J, h=h)), synth.magnetisation_observable(n)).real
    assert abs(m - _mz_dense(n, exact)) < 2e-3


def test_trotter_pin_rejects_sign_mistakes():
    """Planted mistakes in the circuit (the coupling or the field with the
    wrong sign) end far from the exact state, so the pin above catches them."""
    n, J, h, T, steps = 6, 1.0, 0.7, 0.6, 40
    exact = scipy_linalg.expm(-1j * T * _dense_tfim(n, J, h)) @ synth.basis_state(n, 0)
    good = _run(synth.tfim(n, steps, T / steps, J=J, h=h))
    flipped_j = _run(synth.tfim(n, steps, T / steps, J=-J, h=h))
    flipped_h = _run(synth.tfim(n, steps, T / steps, J=J, h=-h))
    base = np.linalg.norm(good - exact)
    assert np.linalg.norm(flipped_j - exact) > 10 * base
    assert np.linalg.norm(flipped_h - exact) > 10 * base
