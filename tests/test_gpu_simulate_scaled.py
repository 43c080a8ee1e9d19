"""Deferred scalars in diaq_simulate (complex128): one-qubit gates whose
rows each hold an entry of the largest magnitude sigma (RX, RY, H) run as
U / sigma with one fused multiply-add per real component, and the last such
gate runs as U times the product of the dropped sigmas. Checked against the
same ops applied one by one and against the FP64 oracle: the TFIM Trotter
circuit, rotations at special angles (cos or sin of either sign, |cos| =
|sin|), a chain of Hadamards long enough that the product falls below
2^-400 and is folded in early, and the state passed in place (psi_in and
psi_out the work buffer). Consecutive one-qubit gates on different qubits
run as one pass (k_apply_pair1), in both precisions."""

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


def test_complex64_pairs_match_op_by_op(api):
    """complex64 circuits of dense one-qubit gates (Haar U(2), RX, H) on
    alternating qubits, paired in one pass, against the same ops one by one."""
    rng = np.random.default_rng(8)
    n = 12
    gates = []
    for i in range(40):
        q = int(rng.integers(n))
        kind = i % 3
        m = synth.random_gate(1, rng, "dense") if kind == 0 else (synth.H if kind == 1 else _rot(q, "X", 0.7).matrix)
        gates.append(synth.Gate((q,), m))
    ops = [api.build(g, n, dtype=torch.complex64) for g in gates]
    psi0 = synth.random_state(n, rng)
    w = torch.as_tensor(psi0).to(torch.complex64).cuda()
    api.simulate(ops, w, w, w)
    x = torch.as_tensor(psi0).to(torch.complex64).cuda()
    for op in ops:
        api.apply(op, x, x)
    assert maxerr(w.cpu().numpy().astype(np.complex128), x.cpu().numpy().astype(np.complex128)) <= 1e-5
    assert maxerr(w.cpu().numpy().astype(np.complex128), _oracle(gates, psi0)) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_diagonal_runs_merge(api, dtype):
    """A long run of diagonal gates (one-, two- and three-qubit phases, CZs,
    controlled phases and a fused six-qubit diagonal op) on 14 qubits is
    merged into passes of at most 11 qubits each; the state matches the same
    ops one by one and the oracle."""
    rng = np.random.default_rng(17)
    n = 14
    gates = [synth.Gate((q,), synth.H) for q in range(n)]
    for i in range(60):
        k = 1 + i % 3
        t = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        if i % 7 == 0:
            m = np.diag([1, 1, 1, -1]).astype(np.complex128)  # CZ: rows untouched
            t = t[:2] if k >= 2 else (t[0], (t[0] + 1) % n)
        elif i % 5 == 0:
            m = np.diag(np.exp(1j * rng.uniform(0, 2 * math.pi, size=1 << k)))
        else:
            m = np.eye(1 << k, dtype=np.complex128)
            m[-1, -1] = np.exp(1j * rng.uniform(0, 2 * math.pi))  # a controlled phase
        gates.append(synth.Gate(t, m))
    gates.append(synth.Gate((3,), synth.H))
    ops = [api.build(g, n, dtype=dtype) for g in gates]
    fused = api.build_fused(gates[n:n + 12], n, 6, 64, dtype=dtype, diagonal=True)
    ops = ops[:n] + fused + ops[n + 12:]
    psi0 = synth.random_state(n, rng)
    w = torch.as_tensor(psi0).to(dtype).cuda()
    api.simulate(ops, w, w, w)
    x = torch.as_tensor(psi0).to(dtype).cuda()
    for op in ops:
        api.apply(op, x, x)
    got = w.cpu().numpy().astype(np.complex128)
    tol = 1e-13 if dtype == torch.complex128 else 1e-5
    assert maxerr(got, x.cpu().numpy().astype(np.complex128)) <= tol
    assert maxerr(got, _oracle(gates, psi0)) <= (TOL_C128 if dtype == torch.complex128 else 1e-5)


def test_simulate_bytes_counts_merges_and_pairs(api):
    """diaq_simulate_bytes: on QFT-12 each run of controlled phases with one
    target b merges into passes of at most 11 qubits that touch the rows with
    bit b set and some control bit of the pass set; H and the SWAPs keep
    their own in-place bytes. Two RX gates on different qubits share one pass."""
    n = 12
    N, s = 1 << n, 16
    circ, _ = synth.qft(n, seed=1)
    ops = [api.build(g, n) for g in circ.gates]
    want = 0
    i = 0
    gates = circ.gates
    while i < len(gates):
        g = gates[i]
        if len(g.targets) == 2 and np.count_nonzero(g.matrix - np.diag(np.diag(g.matrix))) == 0:
            j, qs = i, set(g.targets)
            while j + 1 < len(gates) and len(gates[j + 1].targets) == 2 and \
                    np.count_nonzero(gates[j + 1].matrix - np.diag(np.diag(gates[j + 1].matrix))) == 0 and \
                    len(qs | set(gates[j + 1].targets)) <= 11:
                qs |= set(gates[j + 1].targets)
                j += 1
            if j > i:
                m = len(qs) - 1  # controls of the pass (one common target)
                want += 2 * s * (N // 2) * (1 - 2.0 ** -m)
                i = j + 1
                continue
        want += ops[i].apply_bytes(in_place=True)
        i += 1
    assert api.simulate_bytes(ops) == int(want)
    rx = [api.build(synth.Gate((q,), _rot(q, "X", 0.3).matrix), n) for q in (2, 7)]
    assert api.simulate_bytes(rx) == 2 * N * s
