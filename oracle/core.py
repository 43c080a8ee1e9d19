"""FP64 CPU oracle (test infrastructure only; see the package docstring).

Every function states the passage of arXiv 2405.01250 it follows, or, for
the parts the paper does not cover (expectations, gradients), the
mathematical definition it writes out. The heavy loops run in
``diaq_oracle.c`` (plain C, fp64, no fused multiply-add); numpy's ``matmul``
and ``kron`` serve only as library primitives for dense products.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):

* apply_gate, run_circuit ...... pinned: dense Kronecker matvec (<= 10 qubits),
  GHZ closed form, QFT closed form, norm preservation, paper Fig. 3 / Fig. 5.
* gate_diaq, dense_to_diaq ..... pinned: the paper's 4x4 examples (Section IV
  boxed example, Fig. 5), Fig. 3 offsets, Z gate principal diagonal only.
* diaq_matvec .................. pinned: dense matvec from the same diagonals.
* fuse, embed .................. pinned: unitarity, GHZ-10 fused sparsity
  (>= 99.8 %, Section III-A), equality with sequential application.
* expect, norm2, apply_pauli_sum  pinned: basis-state and |+> special cases,
  GHZ correlators, dense Pauli matrices (<= 8 qubits).
* energy, param_shift_grad ..... pinned: closed-form single-rotation energies
  (RX, RY, RZ), central finite differences, dense-matrix derivative.
* cdf, sample .................. pinned: exact rational inverse-CDF draws on
  states with dyadic probabilities (every sum exact), GHZ and basis-state
  outcomes, zero-probability outcomes never drawn, empirical frequencies
  against |psi|^2 (chi-square), planted mistakes (>= for >, reversed
  order, no normalisation) rejected.
* gate_matrix, pauli_local ..... pinned: scipy.linalg.expm of the full-system
  Pauli operator assembled from X/Z masks, for one- to three-letter
  generators (asymmetric ones included) on non-adjacent and reversed
  targets; a reversed Kronecker order and a flipped sine sign are rejected.
"""

from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build

__all__ = [
    "lib", "threads", "set_threads", "apply_gate", "gate_matrix", "run_circuit",
    "gate_diaq", "dense_to_diaq", "diaq_matvec", "embed", "fuse", "norm2",
    "expect", "apply_pauli_sum", "energy", "param_shift_grad", "fd_grad",
    "fidelity", "max_abs_err", "pauli_local", "cdf", "sample",
]

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i64 = ctypes.c_int64
        i64p = ctypes.POINTER(ctypes.c_int64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_apply_gate.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ip, dp]
        L.oracle_gate_diaq.argtypes = [ctypes.c_int, ctypes.c_int, ip, dp, i64p, i64, dp]
        L.oracle_gate_diaq.restype = i64
        L.oracle_dense_to_diaq.argtypes = [i64, dp, i64p, i64, dp]
        L.oracle_dense_to_diaq.restype = i64
        L.oracle_diaq_matvec.argtypes = [i64, i64, i64p, dp, dp, dp]
        L.oracle_expect.argtypes = [ctypes.c_int, dp, i64, u64p, u64p, dp, dp]
        L.oracle_norm2.argtypes = [ctypes.c_int, dp]
        L.oracle_norm2.restype = ctypes.c_double
        L.oracle_apply_pauli_sum.argtypes = [ctypes.c_int, dp, i64, u64p, u64p, dp, dp]
        L.oracle_cdf.argtypes = [ctypes.c_int, dp, dp]
        L.oracle_sample.argtypes = [ctypes.c_int, dp, i64, dp, i64p]
        _LIB = L
    return _LIB


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(t: int) -> None:
    lib().oracle_set_threads(int(t))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _nq(psi: np.ndarray) -> int:
    n = int(psi.shape[0]).bit_length() - 1
    if psi.ndim != 1 or (1 << n) != psi.shape[0]:
        raise ValueError("state length must be a power of two")
    return n


# --------------------------------------------------------------------------
# Gate application (Section II-C; Algorithm 3 computes the same operator)
# --------------------------------------------------------------------------


def apply_gate(psi, targets, m) -> np.ndarray:
    """(I_above (x) M (x) I_below) psi with the factors on `targets`
    (targets[0] = most significant bit of M's index), by definition, row by
    row. Section II-C; out of place."""
    psi = _c128(psi)
    n = _nq(psi)
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int32))
    k = len(t)
    m = _c128(m)
    if m.shape != (1 << k, 1 << k):
        raise ValueError("gate matrix shape does not match targets")
    if len(set(t.tolist())) != k or (k and (t.min() < 0 or t.max() >= n)):
        raise ValueError("bad targets")
    out = np.empty_like(psi)
    lib().oracle_apply_gate(n, _dp(psi.view(np.float64)), _dp(out.view(np.float64)), k,
                            t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            _dp(m.view(np.float64)))
    return out


_PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def pauli_local(gen: str) -> np.ndarray:
    """Pauli string on a gate's targets as a 2^k x 2^k matrix; the first
    letter acts on targets[0], the most significant local bit, so it is the
    first Kronecker factor."""
    m = np.ones((1, 1), dtype=np.complex128)
    for ch in gen:
        m = np.kron(m, _PAULI[ch.upper()])
    return m


def gate_matrix(gate, theta=None) -> np.ndarray:
    """Matrix of a gate: fixed gates carry theirs; a parametric gate is
    exp(-i a/2 P) = cos(a/2) I - i sin(a/2) P for a Pauli string P (P^2 = I),
    with a = scale * theta[param]."""
    if not gate.parametric:
        return _c128(gate.matrix)
    a = gate.scale * float(theta[gate.param])
    p = pauli_local(gate.gen)
    return math.cos(a / 2) * np.eye(p.shape[0], dtype=np.complex128) - 1j * math.sin(a / 2) * p


def run_circuit(circ, psi0, theta=None) -> np.ndarray:
    """Apply the circuit's gates in order (one time-step per gate)."""
    th = circ.theta if theta is None else theta
    psi = _c128(psi0)
    for g in circ.gates:
        psi = apply_gate(psi, g.targets, gate_matrix(g, th))
    return psi


# --------------------------------------------------------------------------
# DiaQ format (Section IV)
# --------------------------------------------------------------------------


def _unpack(offsets: np.ndarray, flat: np.ndarray, N: int) -> list:
    out, pos = [], 0
    for d in offsets.tolist():
        L = N - abs(d)
        out.append(flat[pos:pos + L].copy())
        pos += L
    return out


def gate_diaq(n: int, targets, m) -> tuple:
    """DiaQ form of a gate's full-system operator: the diagonal indices that
    hold a non-zero element (ascending) and their values, index d >= 0
    holding A[t][t+d], d < 0 holding A[t-d][t] (Algorithm 2's orientation).
    Enumerates all N^2 elements (small n)."""
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int32))
    m = _c128(m)
    k = len(t)
    N = 1 << n
    L = lib()
    tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    cnt = L.oracle_gate_diaq(n, k, tp, _dp(m.view(np.float64)), None, 0, None)
    offs = np.zeros(cnt, dtype=np.int64)
    L.oracle_gate_diaq(n, k, tp, _dp(m.view(np.float64)),
                       offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cnt, None)
    total = int(sum(N - abs(int(d)) for d in offs))
    vals = np.zeros(total, dtype=np.complex128)
    L.oracle_gate_diaq(n, k, tp, _dp(m.view(np.float64)),
                       offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cnt,
                       _dp(vals.view(np.float64)))
    return offs, _unpack(offs, vals, N)


def dense_to_diaq(a) -> tuple:
    """Section IV: DiaQ of a dense square matrix (non-zero diagonals only)."""
    a = _c128(a)
    N = a.shape[0]
    L = lib()
    cnt = L.oracle_dense_to_diaq(N, _dp(a.view(np.float64)), None, 0, None)
    offs = np.zeros(cnt, dtype=np.int64)
    L.oracle_dense_to_diaq(N, _dp(a.view(np.float64)),
                           offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cnt, None)
    total = int(sum(N - abs(int(d)) for d in offs))
    vals = np.zeros(total, dtype=np.complex128)
    L.oracle_dense_to_diaq(N, _dp(a.view(np.float64)),
                           offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cnt,
                           _dp(vals.view(np.float64)))
    return offs, _unpack(offs, vals, N)


def diaq_matvec(offsets, values, x) -> np.ndarray:
    """y = A x for A given by DiaQ diagonals (the product Algorithm 2
    computes), from the definition y[i] = sum_d A[i][i+d] x[i+d]."""
    x = _c128(x)
    N = x.shape[0]
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    for d, v in zip(offs.tolist(), values):
        if len(v) != N - abs(d):
            raise ValueError("diagonal length must be N - |d|")
    flat = _c128(np.concatenate([np.asarray(v) for v in values])) if len(values) else np.zeros(1, np.complex128)
    y = np.empty_like(x)
    lib().oracle_diaq_matvec(N, len(offs), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             _dp(flat.view(np.float64)), _dp(x.view(np.float64)),
                             _dp(y.view(np.float64)))
    return y


def embed(union, targets, m) -> np.ndarray:
    """A gate's matrix on the union target space `union` (union[0] most
    significant). Column C is the gate applied to basis vector e_C of a
    len(union)-qubit register, by the definition of Section II-C."""
    union = list(union)
    K = len(union)
    pos = [K - 1 - union.index(t) for t in targets]
    E = np.zeros((1 << K, 1 << K), dtype=np.complex128)
    for c in range(1 << K):
        e = np.zeros(1 << K, dtype=np.complex128)
        e[c] = 1.0
        E[:, c] = apply_gate(e, pos, m)
    return E


def fuse(gates_with_matrices) -> tuple:
    """Fusion of consecutive gates (Section VI, gate fusion by matrix
    product): returns (union targets, M_last ... M_first) with every gate
    embedded in the union space. Dense product (numpy matmul)."""
    union = []
    for t, _ in gates_with_matrices:
        for q in t:
            if q not in union:
                union.append(q)
    F = np.eye(1 << len(union), dtype=np.complex128)
    for t, m in gates_with_matrices:
        F = embed(union, t, m) @ F
    return tuple(union), F


# --------------------------------------------------------------------------
# Reductions: norm and Pauli-sum expectations (definitions)
# --------------------------------------------------------------------------


def norm2(psi) -> float:
    psi = _c128(psi)
    return float(lib().oracle_norm2(_nq(psi), _dp(psi.view(np.float64))))


def _obs_arrays(obs):
    xm = np.ascontiguousarray(np.asarray(obs.xmask, dtype=np.uint64))
    zm = np.ascontiguousarray(np.asarray(obs.zmask, dtype=np.uint64))
    c = np.asarray(obs.coeff)
    cc = _c128(c.astype(np.complex128) if not np.iscomplexobj(c) else c)
    return xm, zm, cc


def expect(psi, obs) -> complex:
    """<psi| sum_t c_t P_t |psi>, each Pauli string applied factor by factor."""
    psi = _c128(psi)
    xm, zm, cc = _obs_arrays(obs)
    out = np.zeros(2)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib().oracle_expect(_nq(psi), _dp(psi.view(np.float64)), len(xm),
                        xm.ctypes.data_as(u64p), zm.ctypes.data_as(u64p),
                        _dp(cc.view(np.float64) if len(cc) else np.zeros(2)), _dp(out))
    return complex(out[0], out[1])


def apply_pauli_sum(psi, obs) -> np.ndarray:
    """(sum_t c_t P_t) psi, term by term."""
    psi = _c128(psi)
    xm, zm, cc = _obs_arrays(obs)
    lam = np.empty_like(psi)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib().oracle_apply_pauli_sum(_nq(psi), _dp(psi.view(np.float64)), len(xm),
                                 xm.ctypes.data_as(u64p), zm.ctypes.data_as(u64p),
                                 _dp(cc.view(np.float64) if len(cc) else np.zeros(2)),
                                 _dp(lam.view(np.float64)))
    return lam


# --------------------------------------------------------------------------
# Energies and gradients (definitions; the paper has no gradient)
# --------------------------------------------------------------------------


def energy(circ, obs, psi0, theta=None) -> float:
    """E(theta) = Re <psi(theta)| H |psi(theta)>."""
    return expect(run_circuit(circ, psi0, theta), obs).real


def _run_with_angle_override(circ, psi0, theta, gate_idx, delta):
    psi = _c128(psi0)
    for i, g in enumerate(circ.gates):
        if g.parametric:
            a = g.scale * float(theta[g.param]) + (delta if i == gate_idx else 0.0)
            p = pauli_local(g.gen)
            m = math.cos(a / 2) * np.eye(p.shape[0], dtype=np.complex128) - 1j * math.sin(a / 2) * p
        else:
            m = _c128(g.matrix)
        psi = apply_gate(psi, g.targets, m)
    return psi


def param_shift_grad(circ, obs, psi0, theta=None, params=None) -> np.ndarray:
    """dE/dtheta_p by the parameter-shift rule, exact for gates
    exp(-i a/2 P) with P^2 = I: dE/da = [E(a + pi/2) - E(a - pi/2)] / 2 for
    the occurrence's own angle a; by the chain rule a parameter used by
    several gates (angle a = scale * theta_p) collects scale * dE/da over
    its occurrences, in gate order. `params` restricts the evaluation to a
    subset (others are returned as NaN)."""
    th = np.asarray(circ.theta if theta is None else theta, dtype=np.float64)
    want = set(range(len(th))) if params is None else set(int(p) for p in params)
    g = np.full(len(th), np.nan)
    for p in want:
        g[p] = 0.0
    for i, gate in enumerate(circ.gates):
        if not gate.parametric or gate.param not in want:
            continue
        ep = expect(_run_with_angle_override(circ, psi0, th, i, math.pi / 2), obs).real
        em = expect(_run_with_angle_override(circ, psi0, th, i, -math.pi / 2), obs).real
        g[gate.param] += gate.scale * (ep - em) / 2.0
    return g


def fd_grad(circ, obs, psi0, theta=None, h: float = 1e-4, params=None) -> np.ndarray:
    """Central finite differences [E(theta + h e_p) - E(theta - h e_p)] / (2h)."""
    th = np.asarray(circ.theta if theta is None else theta, dtype=np.float64)
    want = range(len(th)) if params is None else params
    g = np.full(len(th), np.nan)
    for p in want:
        tp = th.copy()
        tp[p] += h
        tm = th.copy()
        tm[p] -= h
        g[p] = (energy(circ, obs, psi0, tp) - energy(circ, obs, psi0, tm)) / (2 * h)
    return g


# --------------------------------------------------------------------------
# Shots (Section VII: every benchmark runs 1024 shots): Born-rule sampling
# --------------------------------------------------------------------------


def cdf(psi) -> np.ndarray:
    """cdf_i = sum_{j <= i} |psi_j|^2, summed in index order in FP64."""
    psi = _c128(psi)
    out = np.empty(psi.shape[0], dtype=np.float64)
    lib().oracle_cdf(_nq(psi), _dp(psi.view(np.float64)), _dp(out))
    return out


def sample(psi, uniforms) -> np.ndarray:
    """One basis-state index per uniform u: the smallest i with
    cdf_i > u * cdf_{N-1} (u clamped to [0, 1]; the largest i of non-zero
    probability when none exceeds it; -1 for a zero state)."""
    psi = _c128(psi)
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    out = np.empty(u.shape[0], dtype=np.int64)
    lib().oracle_sample(_nq(psi), _dp(psi.view(np.float64)), u.shape[0], _dp(u),
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


# --------------------------------------------------------------------------
# Error measures used in reports
# --------------------------------------------------------------------------


def fidelity(a, b) -> float:
    """|<a|b>|^2 / (<a|a><b|b>)."""
    a = _c128(a)
    b = _c128(b)
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def max_abs_err(a, b) -> float:
    return float(np.max(np.abs(_c128(a) - _c128(b)))) if len(a) else 0.0
