"""Deferred scalars in diaq_simulate (complex128): one-qubit gates whose
rows each hold an entry of the largest magnitude sigma (RX, RY, H) run as
U / sigma with one fused multiply-add per real component, and the last such
gate runs as U times the product of the dropped sigmas. Checked against the
same ops applied one by one and against the FP64 oracle: the TFIM Trotter
circuit, rotations at special angles (cos or sin of either sign, |cos| =
|sin|), a chain of Hadamards long enough that the product falls below
2^-400 and is folded in early, and the state passed in place (psi_in and
psi_out the work buffer)."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, maxerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _op_by_op(api, ops, psi0):
    x = torch.as_tensor(psi0).cuda()
    for op in ops:
        api.apply(op, x, x)
    return x.cpu().numpy()


def _oracle(gates, psi0, theta=None):
    want = psi0
    for g in gates:
        want = oracle.apply_gate(want, g.targets, oracle.gate_matrix(g, theta))
    return want


def _rot(q, gen, a):
    c, s = math.cos(a / 2), math.sin(a / 2)
    if gen == "X":
        m = np.array([[c, -1j * s], [-1j * s, c]])
    else:
        m = np.array([[c, -s], [s, c]], dtype=np.complex128)
    return synth.Gate((q,), m.astype(np.complex128))


def _check(api, gates, n, psi0, in_place=False, theta=None):
    ops = [api.build(g, n, theta=theta) for g in gates]
    w = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    if in_place:
        w.copy_(torch.as_tensor(psi0))
        api.simulate(ops, w, w, w)
        got = w.cpu().numpy()
    else:
        out = np.empty_like(psi0)
        api.simulate(ops, psi0, out, w)
        got = out
    ref = _op_by_op(api, ops, psi0)
    assert maxerr(got, ref) <= 1e-13
    assert maxerr(got, _oracle(gates, psi0, theta)) <= TOL_C128
    return got


def test_tfim_simulate_matches_op_by_op_and_oracle(api):
    n = 14
    circ = synth.tfim(n, 5, 0.1, J=1.0, h=0.7)
    _check(api, circ.gates, n, synth.basis_state(n, 0), theta=circ.theta)


@pytest.mark.parametrize("in_place", [False, True])
def test_rotations_at_special_angles(api, in_place):
    rng = np.random.default_rng(4)
    n = 10
    q = math.pi / 2
    angles = [0.3, -0.3, q, -q, 3 * q, math.pi - 1e-9, math.pi + 0.2, 2 * math.pi - 0.1, 5.0, 1e-12, 4.0]
    gates = [synth.Gate((i,), synth.H) for i in range(n)]
    for i, a in enumerate(angles * 3):
        gates.append(_rot(int(rng.integers(n)), "XY"[i % 2], a))
        if i % 4 == 3:
            a, b = rng.choice(n, size=2, replace=False)
            gates.append(synth.Gate((int(a), int(b)), synth.CZ))
    _check(api, gates, n, synth.random_state(n, rng), in_place=in_place)


def test_long_hadamard_chain_folds_early(api):
    """Every H has sigma = 1/sqrt(2): after 800 of them the product is below
    2^-400 and the next one is folded in; the state stays exact up to
    rounding."""
    rng = np.random.default_rng(6)
    n = 10
    gates = [synth.Gate((int(q),), synth.H) for q in rng.integers(0, 3, size=1001)]
    gates += [synth.Gate((5,), synth.random_gate(1, rng, "dense"))]
    _check(api, gates, n, synth.random_state(n, rng))
