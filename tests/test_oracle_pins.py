"""Pins for the FP64 oracle against facts that do not come from the oracle:
the paper's printed examples, closed forms, invariants, and brute-force dense
linear algebra written independently here (tensor reshapes and numpy.kron).
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _symbols(grid):
    """Distinct complex numbers for the paper's letters; '0' stays 0."""
    letters = sorted({x for row in grid for x in row if x != "0"})
    val = {s: complex(i + 1, -(i + 1) / 7.0) for i, s in enumerate(letters)}
    return val, np.array([[0 if x == "0" else val[x] for x in row] for row in grid], dtype=np.complex128)


# ---------------------------------------------------------------------------
# Independent dense references
# ---------------------------------------------------------------------------


def dense_apply_tensor(psi, targets, m):
    """Apply m by tensor contraction: psi as an n-axis tensor whose axis a is
    qubit n-1-a (C order, qubit 0 last)."""
    n = int(np.log2(psi.size))
    k = len(targets)
    T = psi.reshape((2,) * n)
    G = m.reshape((2,) * (2 * k))
    axes = [n - 1 - t for t in targets]
    out = np.tensordot(G, T, axes=(list(range(k, 2 * k)), axes))
    # out axes: gate-out axes (targets order), then remaining axes in order
    rest = [a for a in range(n) if a not in axes]
    perm_src = axes + rest
    inv = np.argsort(perm_src)
    return np.transpose(out, inv).reshape(-1)


def dense_full_kron(n, t_low, m):
    """I_above (x) M (x) I_below for contiguous targets t_low+k-1 .. t_low
    (Section II-C), with numpy.kron."""
    k = int(np.log2(m.shape[0]))
    above = np.eye(1 << (n - t_low - k))
    below = np.eye(1 << t_low)
    return np.kron(above, np.kron(m, below))


def dense_pauli(n, xm, zm):
    mats = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Z": np.diag([1, -1]),
            "Y": np.array([[0, -1j], [1j, 0]])}
    P = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):  # most significant qubit is the first factor
        xb, zb = (xm >> q) & 1, (zm >> q) & 1
        ch = "Y" if (xb and zb) else "X" if xb else "Z" if zb else "I"
        P = np.kron(P, mats[ch])
    return P


# ---------------------------------------------------------------------------
# Gate application
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n,k", [(n, k) for n in (1, 3, 6, 9) for k in (1, 2, 3) if k <= n])
def test_apply_gate_matches_tensor_contraction(n, k):
    for trial in range(4):
        targets = [int(t) for t in RNG.choice(n, size=k, replace=False)]
        kind = ["dense", "sparse", "monomial", "diag"][trial % 4]
        m = synth.random_gate(k, RNG, kind)
        psi = synth.random_state(n, RNG)
        np.testing.assert_allclose(oracle.apply_gate(psi, targets, m),
                                   dense_apply_tensor(psi, targets, m), atol=1e-13)


@pytest.mark.parametrize("n,t_low,k", [(4, 0, 1), (4, 3, 1), (6, 2, 2), (7, 4, 3), (10, 3, 2)])
def test_apply_gate_matches_kron_section_iic(n, t_low, k):
    m = synth.random_gate(k, RNG, "dense")
    targets = list(range(t_low + k - 1, t_low - 1, -1))  # MSB first
    psi = synth.random_state(n, RNG)
    A = dense_full_kron(n, t_low, m)
    np.testing.assert_allclose(oracle.apply_gate(psi, targets, m), A @ psi, atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12])
def test_ghz_closed_form(n):
    psi = oracle.run_circuit(synth.ghz(n), synth.basis_state(n, 0))
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) <= 2.3e-16
    assert np.count_nonzero(psi) == 2


def qft_closed_form(n, j):
    N = 1 << n
    k = np.arange(N, dtype=np.uint64)
    ph = ((np.uint64(j) * k) % np.uint64(N)).astype(np.float64) / N
    return np.exp(2j * np.pi * ph) / math.sqrt(N)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 10])
def test_qft_closed_form(n):
    circ, j = synth.qft(n, seed=n)
    psi = oracle.run_circuit(circ, synth.basis_state(n, j))
    assert np.max(np.abs(psi - qft_closed_form(n, j))) < 1e-14


def test_norm_preserved_random_circuit():
    circ = synth.random_layered(8, 6, seed=3)
    psi = oracle.run_circuit(circ, synth.basis_state(8, 0))
    assert abs(oracle.norm2(psi) - 1.0) < 1e-13


# ---------------------------------------------------------------------------
# DiaQ format (Section IV) and gate structure (Section III-A, Fig. 3 / 5)
# ---------------------------------------------------------------------------


def test_section_iv_boxed_example():
    g = _golden("diaq_example_4x4.json")
    val, A = _symbols(g["matrix"])
    offs, vals = oracle.dense_to_diaq(A)
    assert [int(d) for d in offs] == sorted(int(d) for d in g["diaq"])
    for d, v in zip(offs, vals):
        np.testing.assert_array_equal(v, [val[s] for s in g["diaq"][str(int(d))]])


def test_fig5_gate_diagonals():
    g = _golden("gate_application_fig5.json")
    val, G = _symbols(g["gate"])
    # the gate as a 2-qubit operator on a 2-qubit register is the matrix itself
    offs, vals = oracle.gate_diaq(2, [1, 0], G)
    assert [int(d) for d in offs] == sorted(int(d) for d in g["diaq"])
    for d, v in zip(offs, vals):
        np.testing.assert_array_equal(v, [val[s] for s in g["diaq"][str(int(d))]])


def test_fig5_algorithm3_skip_embedding():
    """Algorithm 3 / Fig. 5: in I_dimA (x) G (x) I_dimB each block of
    4*dimB rows (skip = 4*rep*dimB) holds G's diagonals scaled by dimB."""
    g = _golden("gate_application_fig5.json")
    _, G = _symbols(g["gate"])
    n, t_low = 5, 1  # dimB = 2, dimA = 2
    dimB = 1 << t_low
    offs, _ = oracle.gate_diaq(n, [t_low + 1, t_low], G)
    assert sorted(int(d) for d in offs) == sorted(dimB * int(d) for d in g["diaq"])
    x = synth.random_state(n, RNG)
    np.testing.assert_allclose(oracle.apply_gate(x, [t_low + 1, t_low], G),
                               dense_full_kron(n, t_low, G) @ x, atol=1e-12)


def test_fig3_hadamard_offsets_and_z_gate():
    g = _golden("hadamard_patterns_fig3.json")
    n = g["n_qubits"]
    for case in g["cases"]:
        q = int(math.log2(case["i_below"]))
        offs, vals = oracle.gate_diaq(n, [q], synth.H)
        assert [int(d) for d in offs] == case["offsets"]
        # and the same diagonals as the dense Kronecker product
        d_offs, d_vals = oracle.dense_to_diaq(dense_full_kron(n, q, synth.H))
        assert list(d_offs) == list(offs)
        for a, b in zip(vals, d_vals):
            np.testing.assert_array_equal(a, b)
    for q in range(n):
        offs, _ = oracle.gate_diaq(n, [q], np.diag([1, -1]).astype(complex))
        assert [int(d) for d in offs] == g["z_gate_offsets"]


@pytest.mark.parametrize("n,k", [(5, 1), (6, 2), (7, 3)])
def test_gate_diaq_matches_dense_extraction(n, k):
    for kind in ("dense", "sparse", "perm"):
        targets = [int(t) for t in RNG.choice(n, size=k, replace=False)]
        m = synth.random_gate(k, RNG, kind)
        A = np.stack([dense_apply_tensor(np.eye(1 << n)[:, c].astype(complex), targets, m)
                      for c in range(1 << n)], axis=1)
        o1, v1 = oracle.gate_diaq(n, targets, m)
        o2, v2 = oracle.dense_to_diaq(A)
        assert list(o1) == list(o2)
        for a, b in zip(v1, v2):
            np.testing.assert_allclose(a, b, atol=1e-15)


@pytest.mark.parametrize("n,k", [(5, 1), (6, 2), (7, 3), (8, 3)])
def test_row_class_structure_of_gate_diagonals(n, k):
    """A row i whose target bits are c (t[0] most significant) holds, in the
    DiaQ form of a gate, exactly the entries M[c][c2] != 0, on the diagonals
    d = off(c2) - off(c) with off(c) = sum_a bit_a(c) 2^t[a], and zeros on
    every other stored diagonal. (A stored SpMV may therefore give each row
    only the terms of its class, Section II-C's embedding.)"""
    for kind in ("dense", "sparse", "perm", "diag"):
        targets = [int(t) for t in RNG.choice(n, size=k, replace=False)]
        m = synth.random_gate(k, RNG, kind)
        offs, vals = oracle.gate_diaq(n, targets, m)
        K = 1 << k

        def off(c):
            return sum(((c >> (k - 1 - a)) & 1) << targets[a] for a in range(k))

        def local(i):
            return sum(((i >> targets[a]) & 1) << (k - 1 - a) for a in range(k))

        for i in range(1 << n):
            c = local(i)
            want = {off(c2) - off(c): m[c, c2] for c2 in range(K) if m[c, c2] != 0}
            got = {}
            for d, v in zip(offs.tolist(), vals):
                if 0 <= i + d < (1 << n):
                    a = v[i - max(0, -d)]
                    if a != 0:
                        got[d] = a
            assert got == want, (i, c)


def test_embed_matches_kron_with_swaps():
    """Gate matrices on a union target space (union[0] most significant),
    against numpy.kron: adjacent targets are I (x) M (x) I; non-adjacent or
    reversed targets are the adjacent case conjugated by SWAPs."""
    I2 = np.eye(2)
    swap = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    u = [7, 4, 1]  # qubit labels; bit 2, 1, 0 of the local index
    m1 = synth.random_gate(1, RNG, "dense")
    m2 = synth.random_gate(2, RNG, "dense")
    np.testing.assert_allclose(oracle.embed(u, [4], m1), np.kron(np.kron(I2, m1), I2), atol=1e-15)
    np.testing.assert_allclose(oracle.embed(u, [7], m1), np.kron(m1, np.eye(4)), atol=1e-15)
    np.testing.assert_allclose(oracle.embed(u, [7, 4], m2), np.kron(m2, I2), atol=1e-15)
    np.testing.assert_allclose(oracle.embed(u, [4, 1], m2), np.kron(I2, m2), atol=1e-15)
    # targets (7, 1): move qubit 1 next to 7 with a SWAP of the two low bits
    s01 = np.kron(I2, swap)
    np.testing.assert_allclose(oracle.embed(u, [7, 1], m2), s01 @ np.kron(m2, I2) @ s01, atol=1e-15)
    # reversed order (4, 7): the matrix with its two bits exchanged
    np.testing.assert_allclose(oracle.embed(u, [4, 7], m2), np.kron(swap @ m2 @ swap, I2), atol=1e-15)


def test_fidelity_and_error_helpers():
    zero = np.array([1, 0], dtype=complex)
    plus = np.array([1, 1], dtype=complex) / math.sqrt(2)
    one = np.array([0, 1], dtype=complex)
    assert oracle.fidelity(zero, zero) == pytest.approx(1.0)
    assert oracle.fidelity(zero, one) == 0.0
    assert oracle.fidelity(zero, plus) == pytest.approx(0.5)
    assert oracle.fidelity(3j * plus, plus) == pytest.approx(1.0)  # global phase and scale drop out
    assert oracle.max_abs_err(zero, plus) == pytest.approx(1 / math.sqrt(2))  # |0 - 1/sqrt(2)| of amplitude 1
    assert oracle.max_abs_err(np.array([1 + 1j, 2]), np.array([1, 2])) == pytest.approx(1.0)
    assert oracle.max_abs_err(np.array([]), np.array([])) == 0.0


def test_diaq_matvec_matches_dense():
    N = 37  # not a power of two: the DiaQ product is defined for any square matrix
    A = np.zeros((N, N), dtype=np.complex128)
    for d in (-30, -3, 0, 1, 17, 36):
        for i in range(N):
            if 0 <= i + d < N:
                A[i, i + d] = RNG.standard_normal() + 1j * RNG.standard_normal()
    offs, vals = oracle.dense_to_diaq(A)
    x = RNG.standard_normal(N) + 1j * RNG.standard_normal(N)
    np.testing.assert_allclose(oracle.diaq_matvec(offs, vals, x), A @ x, atol=1e-12)


def test_transpose_negates_indices():
    """Section IV: the transpose maps diagonal d to -d with the same values."""
    A = RNG.standard_normal((9, 9)) * (RNG.random((9, 9)) < 0.3)
    o1, v1 = oracle.dense_to_diaq(A.astype(complex))
    o2, v2 = oracle.dense_to_diaq(A.T.astype(complex))
    assert sorted(-int(d) for d in o1) == [int(d) for d in o2]
    m1 = {int(d): v for d, v in zip(o1, v1)}
    for d, v in zip(o2, v2):
        np.testing.assert_array_equal(v, m1[-int(d)])


# ---------------------------------------------------------------------------
# Fusion (matrix product of consecutive gates)
# ---------------------------------------------------------------------------


def test_fuse_equals_sequential_and_is_unitary():
    n = 7
    gates = []
    for _ in range(4):
        k = int(RNG.integers(1, 3))
        t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
        gates.append((t, synth.random_gate(k, RNG, "dense")))
    union, F = oracle.fuse(gates)
    np.testing.assert_allclose(F.conj().T @ F, np.eye(F.shape[0]), atol=1e-13)
    psi = synth.random_state(n, RNG)
    seq = psi
    for t, m in gates:
        seq = oracle.apply_gate(seq, t, m)
    np.testing.assert_allclose(oracle.apply_gate(psi, list(union), F), seq, atol=1e-13)


def test_ghz10_unitary_sparsity_section_iiia():
    g = _golden("ghz10_sparsity.json")
    n = g["n_qubits"]
    N = 1 << n
    circ = synth.ghz(n)
    U = np.eye(N, dtype=np.complex128)
    for gate in circ.gates:
        offs, vals = oracle.gate_diaq(n, gate.targets, gate.matrix)
        step = np.zeros((N, N), dtype=np.complex128)
        for d, v in zip(offs, vals):
            r0, c0 = max(0, -d), max(0, d)
            idx = np.arange(len(v))
            step[r0 + idx, c0 + idx] = v
        U = step @ U
        sparsity = 1.0 - np.count_nonzero(U) / (N * N)
        assert sparsity >= g["min_sparsity"]
    # closed form: permutations times one Hadamard leave exactly 2 non-zeros per column
    assert np.count_nonzero(U) == 2 * N
    # and the fused union-space product agrees with the chained full-system one
    union, F = oracle.fuse([(gt.targets, gt.matrix) for gt in circ.gates])
    e0 = np.zeros(N, dtype=complex)
    e0[0] = 1
    np.testing.assert_allclose(oracle.apply_gate(e0, list(union), F), U[:, 0], atol=1e-15)


# ---------------------------------------------------------------------------
# Norm and Pauli expectations
# ---------------------------------------------------------------------------


def test_expect_basis_and_plus_states():
    n = 5
    for j in (0, 5, 31):
        psi = synth.basis_state(n, j)
        for q in range(n):
            obs = synth.Observable(np.array([0], np.uint64), np.array([1 << q], np.uint64), np.array([1.0]))
            assert oracle.expect(psi, obs) == (-1.0 if (j >> q) & 1 else 1.0)
    plus = np.full(1 << n, 1 / math.sqrt(1 << n), dtype=np.complex128)
    for q in range(n):
        obs = synth.Observable(np.array([1 << q], np.uint64), np.array([0], np.uint64), np.array([1.0]))
        assert abs(oracle.expect(plus, obs) - 1.0) < 1e-15
        obs = synth.Observable(np.array([1 << q], np.uint64), np.array([1 << q], np.uint64), np.array([1.0]))
        assert abs(oracle.expect(plus, obs)) < 1e-15  # <Y> on |+> is 0


def test_expect_ghz_correlators():
    n = 6
    psi = oracle.run_circuit(synth.ghz(n), synth.basis_state(n, 0))
    for i in range(n):
        for j in range(i + 1, n):
            obs = synth.Observable(np.array([0], np.uint64), np.array([(1 << i) | (1 << j)], np.uint64),
                                   np.array([1.0]))
            assert abs(oracle.expect(psi, obs) - 1.0) < 1e-15
    allx = synth.Observable(np.array([(1 << n) - 1], np.uint64), np.array([0], np.uint64), np.array([1.0]))
    assert abs(oracle.expect(psi, allx) - 1.0) < 1e-15


def test_expect_and_pauli_sum_match_dense_pauli_matrices():
    n = 6
    psi = synth.random_state(n, RNG)
    xs = RNG.integers(0, 1 << n, size=7).astype(np.uint64)
    zs = RNG.integers(0, 1 << n, size=7).astype(np.uint64)
    cs = RNG.standard_normal(7)
    obs = synth.Observable(xs, zs, cs)
    Hm = sum(c * dense_pauli(n, int(x), int(z)) for x, z, c in zip(xs, zs, cs))
    assert abs(oracle.expect(psi, obs) - np.vdot(psi, Hm @ psi)) < 1e-13
    np.testing.assert_allclose(oracle.apply_pauli_sum(psi, obs), Hm @ psi, atol=1e-13)
    assert abs(oracle.norm2(psi) - np.vdot(psi, psi).real) < 1e-14
    empty = synth.Observable(np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0))
    assert oracle.expect(psi, empty) == 0


# ---------------------------------------------------------------------------
# Energies and gradients
# ---------------------------------------------------------------------------


def _single_rotation(gen, theta):
    circ = synth.Circuit(1, [synth.Gate((0,), None, param=0, gen=gen)], theta=np.array([theta]))
    return circ


@pytest.mark.parametrize("gen,obs_x,obs_z", [("Y", 0, 1), ("X", 0, 1), ("Y", 1, 0)])
def test_single_rotation_closed_forms(gen, obs_x, obs_z):
    """RY(t)|0>: <Z> = cos t, <X> = sin t; RX(t)|0>: <Z> = cos t."""
    obs = synth.Observable(np.array([obs_x], np.uint64), np.array([obs_z], np.uint64), np.array([1.0]))
    psi0 = synth.basis_state(1, 0)
    for t in (0.0, 0.3, 1.9, 4.0):
        circ = _single_rotation(gen, t)
        e = oracle.energy(circ, obs, psi0)
        de = oracle.param_shift_grad(circ, obs, psi0)[0]
        if obs_z:
            assert abs(e - math.cos(t)) < 1e-15 and abs(de + math.sin(t)) < 1e-15
        else:
            assert abs(e - math.sin(t)) < 1e-15 and abs(de - math.cos(t)) < 1e-15


def test_z_rotation_closed_form():
    """RZ(t)|+> = (e^{-it/2}|0> + e^{it/2}|1>)/sqrt(2): <X> = cos t, <Y> = sin t,
    and the parameter-shift derivatives -sin t, cos t."""
    plus = np.array([1, 1], dtype=np.complex128) / math.sqrt(2)
    ox = synth.Observable(np.array([1], np.uint64), np.array([0], np.uint64), np.array([1.0]))
    oy = synth.Observable(np.array([1], np.uint64), np.array([1], np.uint64), np.array([1.0]))
    for t in (0.0, 0.4, 2.2, 5.1):
        circ = _single_rotation("Z", t)
        assert abs(oracle.energy(circ, ox, plus) - math.cos(t)) < 1e-15
        assert abs(oracle.energy(circ, oy, plus) - math.sin(t)) < 1e-15
        assert abs(oracle.param_shift_grad(circ, ox, plus)[0] + math.sin(t)) < 1e-15
        assert abs(oracle.param_shift_grad(circ, oy, plus)[0] - math.cos(t)) < 1e-15


def _masks_of(gen, targets):
    """(xmask, zmask) of a Pauli string whose letter a acts on qubit targets[a]."""
    return synth.pauli_masks({q: ch for q, ch in zip(targets, gen)})


# Parametric generators on non-adjacent and reversed targets of a 6-qubit
# register, including strings whose letters differ (so a reversed Kronecker
# order changes the operator).
ROTATIONS = [("Z", (4,)), ("X", (1,)), ("Y", (5,)), ("XY", (5, 1)), ("ZX", (0, 3)), ("YZ", (2, 4)),
             ("ZXY", (5, 0, 3)), ("XZ", (1, 0)), ("YX", (3, 5)), ("ZYX", (1, 4, 2))]


def _rotation_pin_error(gen, targets, a, n=6, seed=0):
    """max |oracle - reference| for exp(-i a/2 P) on `targets`, where the
    reference is scipy's matrix exponential of the full-system Pauli
    operator assembled from masks by dense_pauli (numpy.kron over qubits,
    no use of the oracle's pauli_local): once for the gate's local matrix
    (the operator on a k-qubit register, t[0] = its most significant bit)
    and once for its action on a random state."""
    from scipy.linalg import expm
    k = len(targets)
    g = synth.Gate(tuple(targets), None, param=0, gen=gen)
    th = np.array([a])
    m = oracle.gate_matrix(g, th)
    # local register: letter a of gen on local bit k-1-a
    lx, lz = _masks_of(gen, [k - 1 - i for i in range(k)])
    m_ref = expm(-0.5j * a * dense_pauli(k, lx, lz))
    err_local = float(np.max(np.abs(m - m_ref)))
    xm, zm = _masks_of(gen, targets)
    U = expm(-0.5j * a * dense_pauli(n, xm, zm))
    psi = synth.random_state(n, np.random.default_rng(seed))
    err_apply = float(np.max(np.abs(oracle.apply_gate(psi, list(targets), m) - U @ psi)))
    err_tensor = float(np.max(np.abs(dense_apply_tensor(psi, list(targets), m) - U @ psi)))
    return max(err_local, err_apply, err_tensor)


@pytest.mark.parametrize("gen,targets", ROTATIONS)
def test_rotation_matrices_match_expm_of_dense_pauli(gen, targets):
    """Reading R12 (the paper has no rotations): exp(-i a/2 P) for Pauli
    strings on arbitrary target placements, against scipy.linalg.expm."""
    for a in (0.37, 1.9, -2.6, 5.5):
        assert _rotation_pin_error(gen, targets, a) < 1e-13


def test_rotation_pin_rejects_reversed_kronecker_order(monkeypatch):
    """Planted mistake: a pauli_local that takes the Kronecker factors in
    reverse order. The expm pin rejects it for every string whose letters
    differ, and (rightly) cannot tell for palindromes."""
    import oracle.core as core
    good = core.pauli_local

    def reversed_order(gen):
        return good(gen[::-1])

    monkeypatch.setattr(core, "pauli_local", reversed_order)
    for gen, targets in ROTATIONS:
        err = _rotation_pin_error(gen, targets, 1.3)
        if gen != gen[::-1]:
            assert err > 1e-2, (gen, err)
        else:
            assert err < 1e-13
    # a dropped sign of the sine term is rejected for every generator
    monkeypatch.setattr(core, "pauli_local", good)
    monkeypatch.setattr(core, "math", _NegSinMath())
    for gen, targets in ROTATIONS:
        assert _rotation_pin_error(gen, targets, 1.3) > 1e-2, gen


class _NegSinMath:
    """math with sin negated (a planted sign error in exp(-i a/2 P))."""

    def __getattr__(self, name):
        return getattr(math, name)

    @staticmethod
    def sin(x):
        return -math.sin(x)


def _multi_letter_circuit(n=4, seed=9):
    """A small circuit of fixed gates and rotations with multi-letter,
    asymmetric generators on reversed and non-adjacent targets."""
    rng = np.random.default_rng(seed)
    gates = [synth.Gate((0,), synth.H), synth.Gate((2,), synth.H),
             synth.Gate((3, 1), None, param=0, gen="XY"),
             synth.Gate((0, 2), None, param=1, gen="ZX", scale=0.5),
             synth.Gate((1, 3), synth.random_gate(2, rng, "dense")),
             synth.Gate((2, 0, 3), None, param=2, gen="YZX"),
             synth.Gate((1,), None, param=0, gen="Z", scale=-1.5)]
    return synth.Circuit(n, gates, theta=rng.uniform(0, 2 * math.pi, size=3))


@pytest.mark.parametrize("which", ["ansatz", "multi_letter"])
def test_param_shift_vs_fd_and_dense_derivative(which):
    n = 4
    if which == "ansatz":
        circ = synth.ansatz(n=n, layers=2, seed=5)
    else:
        circ = _multi_letter_circuit(n)
    obs = synth.ansatz_observable(n)
    psi0 = synth.basis_state(n, 0)
    g_ps = oracle.param_shift_grad(circ, obs, psi0)
    g_fd = oracle.fd_grad(circ, obs, psi0, h=1e-4)
    assert np.max(np.abs(g_ps - g_fd)) < 1e-6
    # dense derivative: dU/da = -i/2 P U for each occurrence, full matrices,
    # with P the full-system Pauli operator assembled from masks
    N = 1 << n
    Hm = sum(c * dense_pauli(n, int(x), int(z)) for x, z, c in zip(obs.xmask, obs.zmask, obs.coeff))

    def full(g, th):
        return np.stack([dense_apply_tensor(np.eye(N)[:, c].astype(complex), list(g.targets),
                                            oracle.gate_matrix(g, th)) for c in range(N)], axis=1)

    mats = [full(g, circ.theta) for g in circ.gates]
    g_dense = np.zeros(circ.n_params)
    for i, g in enumerate(circ.gates):
        if not g.parametric:
            continue
        P = dense_pauli(n, *_masks_of(g.gen, g.targets))
        U = np.eye(N, dtype=complex)
        dU = np.eye(N, dtype=complex)
        for j, M in enumerate(mats):
            U = M @ U
            dU = (M @ dU) if j != i else (-0.5j * g.scale * P @ M @ dU)
        psi = U @ psi0
        dpsi = dU @ psi0
        g_dense[g.param] += 2 * np.vdot(psi, Hm @ dpsi).real
    assert np.max(np.abs(g_ps - g_dense)) < 1e-12


def test_shared_parameter_chain_rule():
    """A parameter used by several gates (QAOA's gamma_l on every edge) sums
    its occurrences; checked against finite differences."""
    circ, obs = synth.qaoa_instance(6, np.random.default_rng(2), p=2)
    psi0 = synth.basis_state(6, 0)
    g_ps = oracle.param_shift_grad(circ, obs, psi0)
    g_fd = oracle.fd_grad(circ, obs, psi0, h=1e-4)
    assert np.max(np.abs(g_ps - g_fd)) < 1e-6


# ---------------------------------------------------------------------------
# The pins above catch planted mistakes (mutations made here, on the CPU)
# ---------------------------------------------------------------------------


def test_pins_reject_planted_mistakes():
    n = 4
    psi = synth.random_state(n, RNG)
    m = synth.random_gate(2, RNG, "dense")
    good = dense_apply_tensor(psi, [3, 1], m)
    # transposed operand, swapped targets, conjugated matrix: all detected
    assert np.max(np.abs(oracle.apply_gate(psi, [3, 1], m.T) - good)) > 1e-3
    assert np.max(np.abs(oracle.apply_gate(psi, [1, 3], m) - good)) > 1e-3
    assert np.max(np.abs(oracle.apply_gate(psi, [3, 1], m.conj()) - good)) > 1e-3
    # a dropped term in a Pauli sum is detected by the dense reference
    obs = synth.ansatz_observable(n)
    Hm = sum(c * dense_pauli(n, int(x), int(z)) for x, z, c in zip(obs.xmask, obs.zmask, obs.coeff))
    short = synth.Observable(obs.xmask[:-1], obs.zmask[:-1], obs.coeff[:-1])
    assert abs(oracle.expect(psi, short) - np.vdot(psi, Hm @ psi)) > 1e-3
