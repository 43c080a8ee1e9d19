"""Thin Python binding over libdiaq_gb300 (include/diaq.h).

Argument marshalling only: tensors are passed by device pointer with the
current CUDA stream; every step of the gate-apply path runs in the CUDA
library. PyTorch supplies device memory and streams.

Gates are any objects with ``targets``, ``matrix`` (2^k x 2^k complex, or
None for a parametric gate), ``param`` (-1 for fixed), ``gen`` (Pauli letters)
and ``scale`` attributes.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from ._native import DiaqError, check, lib  # noqa: F401

__all__ = [
    "Op", "build", "build_diaq", "fuse", "apply", "simulate", "norm", "expect", "apply_pauli_sum",
    "adjoint_grad", "gate_offsets", "diaq_matmul_host", "fuse_gates_host", "version", "gate_struct",
    "DiaqError", "DiaqEnergy", "Batch", "autotune_apply", "set_apply_launch", "plan_fusion", "autotune_fusion",
    "build_fused", "AdjointPlan", "plan_fusion_commuting", "sample", "shard_schedule", "ShardedState", "plan_fusion_diagonal",
    "ShardRank", "TorchDistTransport",
]


def version() -> str:
    return lib().diaq_version().decode()


def _dtype_code(dtype) -> int:
    if dtype in (torch.complex128, np.complex128, "c128", "complex128"):
        return N.C128
    if dtype in (torch.complex64, np.complex64, "c64", "complex64"):
        return N.C64
    raise ValueError(f"unsupported dtype {dtype}")


def _torch_dtype(code: int):
    return torch.complex128 if code == N.C128 else torch.complex64


def _variant_code(v) -> int:
    if v in ("onthefly", "on_the_fly", N.ONTHEFLY):
        return N.ONTHEFLY
    if v in ("stored", N.STORED):
        return N.STORED
    raise ValueError(f"unknown variant {v}")


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gate_struct(g, keep: list) -> N.diaq_gate:
    """diaq_gate for a gate object; arrays it points to are appended to keep."""
    s = N.diaq_gate()
    t = tuple(int(q) for q in g.targets)
    s.k = len(t)
    if s.k > N.DIAQ_MAX_K:
        raise ValueError(f"gate on {s.k} qubits exceeds {N.DIAQ_MAX_K}")
    for a, q in enumerate(t):
        s.targets[a] = q
    param = int(getattr(g, "param", -1))
    s.param = param
    s.scale = float(getattr(g, "scale", 1.0))
    if param >= 0:
        gen = str(getattr(g, "gen", "")).encode()
        s.gen = gen
        s.m = None
    else:
        m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128))
        keep.append(m)
        s.m = _dptr(m.view(np.float64))
    return s


def _gate_array(gates) -> tuple:
    keep: list = []
    arr = (N.diaq_gate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        arr[i] = gate_struct(g, keep)
    return arr, keep


class Op:
    """Owner of a diaq_op_t (destroyed with the object)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().diaq_op_destroy(h)
            except Exception:
                pass
            self.handle = ctypes.c_void_p(0)

    def close(self):
        self.__del__()

    def info(self) -> dict:
        inf = N.diaq_op_info()
        check(lib().diaq_op_query(self.handle, ctypes.byref(inf)))
        return {
            "n_qubits": inf.n_qubits, "dtype": _torch_dtype(inf.dtype),
            "variant": "stored" if inf.variant == N.STORED else "onthefly",
            "class": N.CLASSES[inf.op_class], "k": inf.k,
            "targets": tuple(inf.targets[a] for a in range(inf.k)),
            "n_diagonals": inf.n_diagonals, "stored_bytes": inf.stored_bytes,
            "real_values": bool(inf.real_values),
        }

    def apply_bytes(self, in_place: bool = False) -> int:
        """Algorithmic HBM bytes of one apply of this op (diaq_op_apply_bytes)."""
        b = ctypes.c_int64(0)
        check(lib().diaq_op_apply_bytes(self.handle, int(bool(in_place)), ctypes.byref(b)))
        return int(b.value)

    def diagonal_nnz(self, stream=None) -> np.ndarray:
        """Values that are not exactly zero, per stored diagonal (index order)."""
        d = int(self.info()["n_diagonals"])
        out = np.zeros(max(d, 1), dtype=np.int64)
        check(lib().diaq_op_diagonal_nnz(self.handle, out.ctypes.data_as(N._i64p), _stream(stream)))
        return out[:d]

    def prune(self, stream=None) -> "Op":
        """A stored copy without its all-zero diagonals (diaq_op_prune)."""
        h = ctypes.c_void_p(0)
        check(lib().diaq_op_prune(self.handle, _stream(stream), ctypes.byref(h)))
        return Op(h.value)

    def offsets(self) -> np.ndarray:
        cnt = ctypes.c_int64(0)
        st = lib().diaq_op_offsets(self.handle, None, 0, ctypes.byref(cnt))
        out = np.zeros(cnt.value, dtype=np.int64)
        check(lib().diaq_op_offsets(self.handle, out.ctypes.data_as(N._i64p), cnt.value, ctypes.byref(cnt)))
        del st
        return out

    def diagonal(self, which: int, stream=None) -> np.ndarray:
        inf = self.info()
        offs = self.offsets()
        L = (1 << inf["n_qubits"]) - abs(int(offs[which]))
        dt = np.complex128 if inf["dtype"] == torch.complex128 else np.complex64
        out = np.zeros(L, dtype=dt)
        check(lib().diaq_op_read_diagonal(self.handle, int(which), out.ctypes.data_as(ctypes.c_void_p),
                                          _stream(stream)))
        return out


def build(gate, n_qubits: int, dtype=torch.complex128, variant="onthefly", theta=None, stream=None) -> Op:
    keep: list = []
    s = gate_struct(gate, keep)
    th = None
    if theta is not None:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        keep.append(th)
    h = ctypes.c_void_p(0)
    check(lib().diaq_build(ctypes.byref(s), int(n_qubits), _dtype_code(dtype), _variant_code(variant),
                           _dptr(th) if th is not None else None, _stream(stream), ctypes.byref(h)))
    return Op(h.value)


def build_diaq(n_qubits: int, indices, values, dtype=torch.complex128, stream=None) -> Op:
    idx = np.ascontiguousarray(np.asarray(indices, dtype=np.int64))
    vals = [np.asarray(v, dtype=np.complex128) for v in values]
    flat = np.ascontiguousarray(np.concatenate(vals)) if vals else np.zeros(1, np.complex128)
    h = ctypes.c_void_p(0)
    check(lib().diaq_build_diaq(int(n_qubits), len(idx), idx.ctypes.data_as(N._i64p), _dptr(flat.view(np.float64)),
                                _dtype_code(dtype), _stream(stream), ctypes.byref(h)))
    return Op(h.value)


def fuse(ops, variant="onthefly", stream=None) -> Op:
    arr = (ctypes.c_void_p * len(ops))(*[o.handle.value for o in ops])
    h = ctypes.c_void_p(0)
    check(lib().diaq_fuse(arr, len(ops), _variant_code(variant), _stream(stream), ctypes.byref(h)))
    return Op(h.value)


def _check_state(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if t.dtype not in (torch.complex64, torch.complex128):
        raise ValueError(f"{name} must be complex64 or complex128")


def _nq(t: torch.Tensor) -> int:
    n = int(t.numel()).bit_length() - 1
    if (1 << n) != t.numel():
        raise ValueError("state length must be a power of two")
    return n


def apply(op: Op, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y = A x (y may be x for on-the-fly ops)."""
    _check_state(x, "x")
    _check_state(y, "y")
    check(lib().diaq_apply(op.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), _stream(stream)))
    return y


def _ptr(t) -> ctypes.c_void_p:
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def inject_alloc_failure(after: int) -> None:
    """Testing hook: the after-th next library allocation fails (-1: off)."""
    check(lib().diaq_debug_inject_alloc_failure(int(after)))


def unitary_chain(gates, n_qubits: int, dtype=torch.complex128, theta=None, prune: bool = True, stream=None):
    """Unitary of a circuit by chained device DiaQ products (diaq_unitary_chain).
    Returns (op, diagonals per time step, non-zeros per time step)."""
    arr, keep = _gate_array(gates)
    th = np.ascontiguousarray(np.asarray(theta if theta is not None else [0.0], dtype=np.float64))
    nd = np.zeros(len(gates), dtype=np.int64)
    nz = np.zeros(len(gates), dtype=np.int64)
    h = ctypes.c_void_p(0)
    check(lib().diaq_unitary_chain(arr, len(gates), _dptr(th), int(n_qubits), _dtype_code(dtype), int(bool(prune)),
                                   nd.ctypes.data_as(N._i64p), nz.ctypes.data_as(N._i64p), _stream(stream),
                                   ctypes.byref(h)))
    del keep
    return Op(h.value), nd, nz


def simulate(ops, psi_in, psi_out, work0: torch.Tensor, work1: torch.Tensor | None = None, stream=None,
             timeline: bool = False):
    """Run ops in order; psi_in / psi_out may be host (numpy / CPU tensor) or
    device. With timeline=True returns (psi_out, [input copied, last op done,
    output copied] in ms from the start of the call's device work)."""
    arr = (ctypes.c_void_p * len(ops))(*[o.handle.value for o in ops])
    tl = (ctypes.c_float * 3)()
    check(lib().diaq_simulate_timed(arr, len(ops), _ptr(psi_in), _ptr(psi_out), _ptr(work0),
                                    _ptr(work1) if work1 is not None else None, _stream(stream),
                                    tl if timeline else None))
    return (psi_out, [tl[0], tl[1], tl[2]]) if timeline else psi_out


def simulate_bytes(ops) -> int:
    """HBM bytes that simulate moves for ops on a device state (diaq_simulate_bytes)."""
    arr = (ctypes.c_void_p * len(ops))(*[o.handle.value for o in ops])
    b = ctypes.c_int64(0)
    check(lib().diaq_simulate_bytes(arr, len(ops), ctypes.byref(b)))
    return int(b.value)


def norm(psi: torch.Tensor, stream=None) -> float:
    _check_state(psi, "psi")
    out = ctypes.c_double(0)
    check(lib().diaq_norm(ctypes.c_void_p(psi.data_ptr()), _nq(psi), _dtype_code(psi.dtype), ctypes.byref(out),
                          _stream(stream)))
    return out.value


def sample(psi: torch.Tensor, uniforms, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Born-rule shots of psi (diaq_sample): one basis-state index per
    uniform in [0, 1). uniforms: a float64 CUDA tensor, or host values that
    are copied to the device first. Returns a CUDA int64 tensor."""
    _check_state(psi, "psi")
    if not (isinstance(uniforms, torch.Tensor) and uniforms.is_cuda):
        uniforms = torch.as_tensor(np.asarray(uniforms, dtype=np.float64)).to(psi.device)
    if uniforms.dtype != torch.float64 or not uniforms.is_contiguous():
        raise ValueError("uniforms must be a contiguous float64 tensor")
    shots = uniforms.numel()
    if out is None:
        out = torch.empty(shots, dtype=torch.int64, device=psi.device)
    if out.dtype != torch.int64 or out.numel() != shots or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous CUDA int64 tensor with one entry per uniform")
    check(lib().diaq_sample(ctypes.c_void_p(psi.data_ptr()), _nq(psi), _dtype_code(psi.dtype),
                            ctypes.c_void_p(uniforms.data_ptr()), shots, ctypes.c_void_p(out.data_ptr()),
                            _stream(stream)))
    return out


def _terms(xmask, zmask, coeff):
    xm = np.ascontiguousarray(np.asarray(xmask, dtype=np.uint64))
    zm = np.ascontiguousarray(np.asarray(zmask, dtype=np.uint64))
    c = np.ascontiguousarray(np.asarray(coeff).astype(np.complex128))
    if not (len(xm) == len(zm) == len(c)):
        raise ValueError("xmask, zmask and coeff must have one entry per term")
    return xm, zm, c


def expect(psi: torch.Tensor, xmask, zmask, coeff, stream=None) -> complex:
    _check_state(psi, "psi")
    xm, zm, c = _terms(xmask, zmask, coeff)
    out = (ctypes.c_double * 2)()
    check(lib().diaq_expect(ctypes.c_void_p(psi.data_ptr()), _nq(psi), _dtype_code(psi.dtype), len(xm),
                            xm.ctypes.data_as(N._u64p), zm.ctypes.data_as(N._u64p),
                            _dptr(c.view(np.float64)) if len(c) else None, out, _stream(stream)))
    return complex(out[0], out[1])


def apply_pauli_sum(psi: torch.Tensor, lam: torch.Tensor, xmask, zmask, coeff, stream=None) -> torch.Tensor:
    _check_state(psi, "psi")
    _check_state(lam, "lam")
    xm, zm, c = _terms(xmask, zmask, coeff)
    check(lib().diaq_apply_pauli_sum(ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(lam.data_ptr()), _nq(psi),
                                     _dtype_code(psi.dtype), len(xm), xm.ctypes.data_as(N._u64p),
                                     zm.ctypes.data_as(N._u64p), _dptr(c.view(np.float64)) if len(c) else None,
                                     _stream(stream)))
    return lam


def adjoint_grad(gates, theta, xmask, zmask, coeff, psi0: torch.Tensor, work_psi: torch.Tensor,
                 work_lam: torch.Tensor, stream=None) -> tuple:
    """(energy, gradient) of <psi(theta)|H|psi(theta)> by one adjoint sweep."""
    for t, nm in ((psi0, "psi0"), (work_psi, "work_psi"), (work_lam, "work_lam")):
        _check_state(t, nm)
    arr, keep = _gate_array(gates)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    xm, zm, c = _terms(xmask, zmask, coeff)
    grad = np.zeros(len(th), dtype=np.float64)
    e = ctypes.c_double(0)
    check(lib().diaq_adjoint_grad(arr, len(gates), _dptr(th) if len(th) else None, len(th), len(xm),
                                  xm.ctypes.data_as(N._u64p), zm.ctypes.data_as(N._u64p),
                                  _dptr(c.view(np.float64)) if len(c) else None,
                                  ctypes.c_void_p(psi0.data_ptr()), ctypes.c_void_p(work_psi.data_ptr()),
                                  ctypes.c_void_p(work_lam.data_ptr()), _nq(psi0), _dtype_code(psi0.dtype),
                                  ctypes.byref(e), _dptr(grad) if len(grad) else None, _stream(stream)))
    del keep
    return e.value, grad


def gate_offsets(gate, n_qubits: int) -> np.ndarray:
    keep: list = []
    s = gate_struct(gate, keep)
    cnt = ctypes.c_int64(0)
    lib().diaq_gate_offsets(ctypes.byref(s), int(n_qubits), None, 0, ctypes.byref(cnt))
    out = np.zeros(max(cnt.value, 1), dtype=np.int64)
    check(lib().diaq_gate_offsets(ctypes.byref(s), int(n_qubits), out.ctypes.data_as(N._i64p), len(out),
                                  ctypes.byref(cnt)))
    return out[:cnt.value]


def diaq_matmul_host(Nord: int, a_idx, a_vals, b_idx, b_vals) -> tuple:
    """Host DiaQ product C = A B (Algorithm 1). Values are lists of arrays."""
    def pack(idx, vals):
        i = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        v = np.ascontiguousarray(np.concatenate([np.asarray(x, np.complex128) for x in vals])) if len(vals) \
            else np.zeros(1, np.complex128)
        return i, v
    ai, av = pack(a_idx, a_vals)
    bi, bv = pack(b_idx, b_vals)
    cc = ctypes.c_int64(0)
    cl = ctypes.c_int64(0)
    L = lib()
    check(L.diaq_diaq_matmul_host(Nord, len(ai), ai.ctypes.data_as(N._i64p), _dptr(av.view(np.float64)),
                                  len(bi), bi.ctypes.data_as(N._i64p), _dptr(bv.view(np.float64)),
                                  ctypes.byref(cc), None, ctypes.byref(cl), None))
    ci = np.zeros(max(cc.value, 1), np.int64)
    cv = np.zeros(max(cl.value, 1), np.complex128)
    check(L.diaq_diaq_matmul_host(Nord, len(ai), ai.ctypes.data_as(N._i64p), _dptr(av.view(np.float64)),
                                  len(bi), bi.ctypes.data_as(N._i64p), _dptr(bv.view(np.float64)),
                                  ctypes.byref(cc), ci.ctypes.data_as(N._i64p), ctypes.byref(cl),
                                  _dptr(cv.view(np.float64))))
    out, pos = [], 0
    for d in ci[:cc.value]:
        n = Nord - abs(int(d))
        out.append(cv[pos:pos + n].copy())
        pos += n
    return ci[:cc.value], out


def fuse_gates_host(gates, theta=None) -> tuple:
    """(union targets, fused 2^K x 2^K matrix) of gates[-1] ... gates[0]."""
    arr, keep = _gate_array(gates)
    th = None if theta is None else np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    uk = ctypes.c_int32(0)
    ut = (ctypes.c_int32 * N.DIAQ_MAX_K)()
    fm = np.zeros(2 * (1 << (2 * N.DIAQ_MAX_K)), dtype=np.float64)
    check(lib().diaq_fuse_gates_host(arr, len(gates), _dptr(th) if th is not None else None, ctypes.byref(uk), ut,
                                     _dptr(fm)))
    K = uk.value
    m = fm[: 2 * (1 << (2 * K))].view(np.complex128).reshape(1 << K, 1 << K).copy()
    del keep
    return tuple(ut[a] for a in range(K)), m


def autotune_apply(n_qubits: int, x: torch.Tensor, y: torch.Tensor, reps: int = 3, stream=None) -> dict:
    """Pick the on-the-fly launch shape per k (process-wide) by timing."""
    _check_state(x, "x")
    _check_state(y, "y")
    rep = N.diaq_apply_tuning()
    check(lib().diaq_autotune_apply(int(n_qubits), _dtype_code(x.dtype), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), int(reps), ctypes.byref(rep), _stream(stream)))
    return {"rows": [(rep.k[i], rep.threads[i], rep.groups[i], rep.ms[i]) for i in range(rep.n_rows)],
            "best": {k + 1: (rep.best_threads[k], rep.best_groups[k], rep.best_ms[k]) for k in range(3)}}


def set_apply_launch(dtype, k: int, threads: int, groups: int) -> None:
    check(lib().diaq_set_apply_launch(_dtype_code(dtype), int(k), int(threads), int(groups)))


def plan_fusion(gates, max_k: int, max_depth: int) -> list:
    """Group index of each gate for fusion (consecutive groups)."""
    arr, keep = _gate_array(gates)
    out = np.zeros(max(1, len(gates)), dtype=np.int32)
    ng = ctypes.c_int32(0)
    check(lib().diaq_plan_fusion(arr, len(gates), int(max_k), int(max_depth), out.ctypes.data_as(N._i32p),
                                 ctypes.byref(ng)))
    del keep
    return out[:len(gates)].tolist()


def plan_fusion_commuting(gates, max_k: int, max_depth: int) -> tuple:
    """(execution order, group of each position) with gates moved past
    commuting gates (disjoint qubits) into earlier groups."""
    arr, keep = _gate_array(gates)
    order = np.zeros(max(1, len(gates)), dtype=np.int32)
    grp = np.zeros(max(1, len(gates)), dtype=np.int32)
    ng = ctypes.c_int32(0)
    check(lib().diaq_plan_fusion_commuting(arr, len(gates), int(max_k), int(max_depth), order.ctypes.data_as(N._i32p),
                                           grp.ctypes.data_as(N._i32p), ctypes.byref(ng)))
    del keep
    return order[:len(gates)].tolist(), grp[:len(gates)].tolist()


def plan_fusion_diagonal(gates, max_k: int, max_depth: int) -> list:
    """Group index per gate: runs of diagonal gates fuse, other gates stay
    alone (diaq_plan_fusion_diagonal)."""
    arr, keep = _gate_array(gates)
    grp = np.zeros(max(1, len(gates)), dtype=np.int32)
    ng = ctypes.c_int32(0)
    check(lib().diaq_plan_fusion_diagonal(arr, len(gates), max_k, max_depth, grp.ctypes.data_as(N._i32p),
                                          ctypes.byref(ng)))
    return grp[: len(gates)].tolist()


def build_fused(gates, n_qubits: int, max_k: int, max_depth: int, dtype=torch.complex128, variant="onthefly",
                theta=None, stream=None, commuting: bool = False, diagonal: bool = False) -> list:
    """Ops for a circuit with gates fused per plan_fusion (consecutive
    groups), per plan_fusion_commuting (commuting=True) or per
    plan_fusion_diagonal (diagonal=True: runs of diagonal gates only)."""
    if commuting:
        order, grp = plan_fusion_commuting(gates, max_k, max_depth)
        gates = [gates[i] for i in order]
    elif diagonal:
        grp = plan_fusion_diagonal(gates, max_k, max_depth)
    else:
        grp = plan_fusion(gates, max_k, max_depth)
    ops, i = [], 0
    while i < len(gates):
        j = i
        while j < len(gates) and grp[j] == grp[i]:
            j += 1
        part = [build(g, n_qubits, dtype=dtype, variant="onthefly", theta=theta, stream=stream) for g in gates[i:j]]
        if len(part) == 1 and variant == "onthefly":
            ops.append(part[0])
        else:
            ops.append(fuse(part, variant=variant, stream=stream))
        i = j
    return ops


def autotune_fusion(gates, n_qubits: int, work: torch.Tensor, max_k: int = 4, max_depth: int = 4, theta=None,
                    stream=None, commuting: bool = False) -> dict:
    _check_state(work, "work")
    arr, keep = _gate_array(gates)
    th = None if theta is None else np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    rep = N.diaq_fusion_tuning()
    check(lib().diaq_autotune_fusion(arr, len(gates), _dptr(th) if th is not None else None, int(n_qubits),
                                     _dtype_code(work.dtype), ctypes.c_void_p(work.data_ptr()), int(max_k),
                                     int(max_depth), int(bool(commuting)), ctypes.byref(rep), _stream(stream)))
    del keep
    return {"ops": [rep.ops[d] for d in range(rep.n_depths)], "ms": [rep.ms[d] for d in range(rep.n_depths)],
            "best_depth": rep.best_depth}


class AdjointPlan:
    """The adjoint sweep of one circuit recorded as a CUDA graph
    (diaq_adjoint_plan_*), replayed for each theta."""

    def __init__(self, gates, n_params: int, observable, n_qubits: int, dtype=torch.complex128):
        arr, keep = _gate_array(gates)
        xm, zm, c = _terms(*observable)
        h = ctypes.c_void_p(0)
        check(lib().diaq_adjoint_plan_create(arr, len(gates), int(n_params), len(xm), xm.ctypes.data_as(N._u64p),
                                             zm.ctypes.data_as(N._u64p),
                                             _dptr(c.view(np.float64)) if len(c) else None, int(n_qubits),
                                             _dtype_code(dtype), ctypes.byref(h)))
        del keep
        self.handle = h
        self.n_params = int(n_params)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().diaq_adjoint_plan_destroy(h)
            except Exception:
                pass
            self.handle = ctypes.c_void_p(0)

    def close(self):
        self.__del__()

    def run(self, theta, psi0: torch.Tensor | None = None, stream=None) -> tuple:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if len(th) != self.n_params:
            raise ValueError("theta length does not match the plan")
        g = np.zeros(max(1, self.n_params))
        e = ctypes.c_double(0)
        check(lib().diaq_adjoint_plan_run(self.handle, _dptr(th) if len(th) else None,
                                          ctypes.c_void_p(psi0.data_ptr()) if psi0 is not None else None,
                                          ctypes.byref(e), _dptr(g), _stream(stream)))
        return e.value, g[:self.n_params].copy()

    def set_window(self, window: int) -> None:
        """0: one launch per gate; 2..5: window-fused blocks (diaq_adjoint_plan_set_window)."""
        check(lib().diaq_adjoint_plan_set_window(self.handle, int(window)))

    def autotune(self, theta, reps: int = 3) -> dict:
        """Time windows 0, 3, 4, 5 and keep the fastest (diaq_adjoint_plan_autotune)."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        rep = N.diaq_plan_tuning()
        check(lib().diaq_adjoint_plan_autotune(self.handle, _dptr(th) if len(th) else None, int(reps),
                                               ctypes.byref(rep)))
        return {"tried": [(rep.window[i], rep.lanes[i], rep.blocks[i], rep.ms[i]) for i in range(rep.n_tried)],
                "best_window": rep.best_window, "best_lanes": rep.best_lanes, "best_blocks": rep.best_blocks,
                "best_ms": rep.best_ms}

    def set_blocks(self, blocks: int) -> None:
        """Blocks of the per-gate sweep's kernels; 0 = two per SM (diaq_adjoint_plan_set_blocks)."""
        check(lib().diaq_adjoint_plan_set_blocks(self.handle, int(blocks)))

    def blocks(self) -> int:
        a = ctypes.c_int32(0)
        check(lib().diaq_adjoint_plan_get_blocks(self.handle, ctypes.byref(a)))
        return int(a.value)

    def set_sweep(self, window: int, lanes: int) -> None:
        """window 0 (per gate) or 2..5, with 1 or 4 threads per group (diaq_adjoint_plan_set_sweep)."""
        check(lib().diaq_adjoint_plan_set_sweep(self.handle, int(window), int(lanes)))

    def set_runs(self, on: bool) -> None:
        """Diagonal runs of the per-gate sweep on or off (diaq_adjoint_plan_set_runs)."""
        check(lib().diaq_adjoint_plan_set_runs(self.handle, int(bool(on))))

    def set_scaled(self, on: bool) -> None:
        """Scaled rotations of the per-gate complex128 sweep on or off (diaq_adjoint_plan_set_scaled)."""
        check(lib().diaq_adjoint_plan_set_scaled(self.handle, int(bool(on))))

    def set_pairs(self, on: bool) -> None:
        """Fused one-qubit rotation pairs of the per-gate sweep on or off (diaq_adjoint_plan_set_pairs)."""
        check(lib().diaq_adjoint_plan_set_pairs(self.handle, int(bool(on))))

    def pairs(self) -> bool:
        a = ctypes.c_int32(0)
        check(lib().diaq_adjoint_plan_get_pairs(self.handle, ctypes.byref(a)))
        return bool(a.value)

    def scaled(self) -> tuple:
        """(requested, active) for the scaled rotations (diaq_adjoint_plan_get_scaled)."""
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        check(lib().diaq_adjoint_plan_get_scaled(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return bool(a.value), bool(b.value)

    def runs(self) -> tuple:
        """(on, runs in the circuit, launches per sweep direction)."""
        a, b, c = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        check(lib().diaq_adjoint_plan_get_runs(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return bool(a.value), b.value, c.value

    def sweep(self) -> tuple:
        """(window, lanes, launches per sweep)."""
        w, ln, nb = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        check(lib().diaq_adjoint_plan_get_sweep(self.handle, ctypes.byref(w), ctypes.byref(ln), ctypes.byref(nb)))
        return w.value, ln.value, nb.value

    def window(self) -> tuple:
        """(window, launches per sweep)."""
        w = ctypes.c_int32(0)
        nb = ctypes.c_int32(0)
        check(lib().diaq_adjoint_plan_get_window(self.handle, ctypes.byref(w), ctypes.byref(nb)))
        return w.value, nb.value


class Batch:
    """Energies and adjoint gradients of many circuits (uneven qubit counts)
    in one persistent launch replayed from a CUDA graph (diaq_batch_*).

    instances: list of (n_qubits, gates, n_params, (xmask, zmask, coeff));
    every circuit starts from |0...0>."""

    def __init__(self, instances, dtype=torch.complex128):
        nq, gfirst, pfirst, tfirst = [], [0], [0], [0]
        gates, xs, zs, cs = [], [], [], []
        for n, gl, npar, (xm, zm, co) in instances:
            nq.append(int(n))
            gates.extend(gl)
            gfirst.append(len(gates))
            pfirst.append(pfirst[-1] + int(npar))
            x, z, c = _terms(xm, zm, co)
            xs.append(x)
            zs.append(z)
            cs.append(c)
            tfirst.append(tfirst[-1] + len(x))
        self.n_inst = len(nq)
        self.param_first = list(pfirst)
        arr, keep = _gate_array(gates)
        i32 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.int32))  # noqa: E731
        nq_a, gf_a, pf_a, tf_a = i32(nq), i32(gfirst), i32(pfirst), i32(tfirst)
        xm = np.ascontiguousarray(np.concatenate(xs) if xs else np.zeros(0, np.uint64))
        zm = np.ascontiguousarray(np.concatenate(zs) if zs else np.zeros(0, np.uint64))
        co = np.ascontiguousarray(np.concatenate(cs) if cs else np.zeros(0, np.complex128))
        h = ctypes.c_void_p(0)
        p32 = N._i32p
        check(lib().diaq_batch_create(self.n_inst, nq_a.ctypes.data_as(p32), gf_a.ctypes.data_as(p32), arr,
                                      pf_a.ctypes.data_as(p32), tf_a.ctypes.data_as(p32),
                                      xm.ctypes.data_as(N._u64p), zm.ctypes.data_as(N._u64p),
                                      _dptr(co.view(np.float64)) if len(co) else None, _dtype_code(dtype),
                                      ctypes.byref(h)))
        del keep
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().diaq_batch_destroy(h)
            except Exception:
                pass
            self.handle = ctypes.c_void_p(0)

    def close(self):
        self.__del__()

    def run(self, theta, stream=None) -> tuple:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        if len(th) != self.param_first[-1]:
            raise ValueError(f"theta has {len(th)} values, the batch has {self.param_first[-1]} parameters")
        e = np.zeros(self.n_inst)
        g = np.zeros(max(1, len(th)))
        check(lib().diaq_batch_run(self.handle, _dptr(th) if len(th) else None, _dptr(e), _dptr(g), _stream(stream)))
        return e, [g[self.param_first[i]:self.param_first[i + 1]].copy() for i in range(self.n_inst)]

    def set_launch(self, cluster: int, threads: int):
        check(lib().diaq_batch_set_launch(self.handle, int(cluster), int(threads)))

    def autotune(self, theta, reps: int = 2, stream=None) -> dict:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        rep = N.diaq_batch_tuning()
        check(lib().diaq_batch_autotune(self.handle, _dptr(th) if len(th) else None, int(reps), ctypes.byref(rep),
                                        _stream(stream)))
        return {"tried": [(rep.cluster[i], rep.threads[i], rep.window[i], rep.lanes[i], rep.ms[i])
                          for i in range(rep.n_tried)],
                "best_cluster": rep.best_cluster, "best_threads": rep.best_threads, "best_window": rep.best_window,
                "best_lanes": rep.best_lanes, "best_ms": rep.best_ms}

    def set_sweep(self, window: int, lanes: int):
        """window 0 or 2..5, with 1 or 4 threads per group (diaq_batch_set_sweep)."""
        check(lib().diaq_batch_set_sweep(self.handle, int(window), int(lanes)))

    def sweep(self) -> tuple:
        w, ln = ctypes.c_int32(0), ctypes.c_int32(0)
        check(lib().diaq_batch_get_sweep(self.handle, ctypes.byref(w), ctypes.byref(ln)))
        return w.value, ln.value

    def set_runs(self, on: bool):
        """Diagonal runs of the per-gate team kernel on or off (diaq_batch_set_runs)."""
        check(lib().diaq_batch_set_runs(self.handle, int(bool(on))))

    def set_scaled(self, on: bool):
        """Scaled rotations of the per-gate complex128 team kernel on or off (diaq_batch_set_scaled)."""
        check(lib().diaq_batch_set_scaled(self.handle, int(bool(on))))

    def scaled(self) -> tuple:
        """(requested, active) for the scaled rotations (diaq_batch_get_scaled)."""
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        check(lib().diaq_batch_get_scaled(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return bool(a.value), bool(b.value)

    def runs(self) -> tuple:
        """(on, diagonal runs in the batch's circuits)."""
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        check(lib().diaq_batch_get_runs(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return bool(a.value), b.value

    def set_window(self, window: int):
        """0: one pass per gate; 2..5: window-fused blocks (diaq_batch_set_window)."""
        check(lib().diaq_batch_set_window(self.handle, int(window)))

    def window(self) -> int:
        w = ctypes.c_int32(0)
        check(lib().diaq_batch_get_window(self.handle, ctypes.byref(w)))
        return w.value

    def query(self) -> dict:
        c, t, tm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ab = ctypes.c_int64()
        check(lib().diaq_batch_query(self.handle, ctypes.byref(c), ctypes.byref(t), ctypes.byref(tm), ctypes.byref(ab)))
        return {"cluster": c.value, "threads": t.value, "teams": tm.value, "arena_bytes": ab.value}


class DiaqEnergy(torch.autograd.Function):
    """E(theta) = <psi(theta)|H|psi(theta)> with the gradient from the
    adjoint sweep. Call as DiaqEnergy.apply(theta, gates, (xmask, zmask,
    coeff), psi0) (diaq_adjoint_grad, one launch per gate), or as
    DiaqEnergy.apply(theta, plan, None, psi0_or_None) with an AdjointPlan
    (the graph-recorded sweep)."""

    @staticmethod
    def forward(ctx, theta, gates, observable, psi0):
        th = theta.detach().cpu().numpy()
        if isinstance(gates, AdjointPlan):
            e, g = gates.run(th, psi0)
        else:
            xm, zm, c = observable
            work_psi = torch.empty_like(psi0)
            work_lam = torch.empty_like(psi0)
            e, g = adjoint_grad(gates, th, xm, zm, c, psi0, work_psi, work_lam)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return theta.new_tensor(e)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None


# ---------------------------------------------------------------------------
# Sharded state (diaq_shard_* / diaq_sharded_*): 2^g shards split by the top
# g bits of the physical basis index, qubits remapped by exchanges.
# ---------------------------------------------------------------------------


def shard_schedule(gates, n_qubits: int, global_bits: int, restore: bool = True) -> tuple:
    """Step list of diaq_shard_schedule as dicts, and the final map
    (physical bit of each logical qubit). Host only."""
    arr, keep = _gate_array(gates)
    cnt = ctypes.c_int32(0)
    check(lib().diaq_shard_schedule(arr, len(gates), n_qubits, global_bits, int(bool(restore)), None, 0,
                                    ctypes.byref(cnt), None))
    steps = (N.diaq_shard_step * max(1, cnt.value))()
    fmap = (ctypes.c_int32 * n_qubits)()
    check(lib().diaq_shard_schedule(arr, len(gates), n_qubits, global_bits, int(bool(restore)), steps, cnt.value,
                                    ctypes.byref(cnt), fmap))
    out = []
    for i in range(cnt.value):
        s = steps[i]
        out.append({"kind": ("apply", "exchange", "local_swap")[s.kind], "gate": s.gate,
                    "targets": tuple(s.targets[a] for a in range(s.k)), "global_bit": s.global_bit,
                    "local_bit": s.local_bit})
    return out, list(fmap)


def _shard_ptrs(shards):
    return (ctypes.c_void_p * len(shards))(*[t.data_ptr() for t in shards])


class ShardedState:
    """2^global_bits shards of one state on the current device (one process),
    each a CUDA tensor of 2^(n - global_bits) amplitudes. Shard s holds the
    physical indices s 2^(n-g) .. (s+1) 2^(n-g) - 1; `map` gives the physical
    bit of each logical qubit (identity after a run with restore)."""

    def __init__(self, n_qubits: int, global_bits: int, dtype=torch.complex128, shards=None):
        self.n, self.g = int(n_qubits), int(global_bits)
        self.n_local = self.n - self.g
        self.dtype = dtype
        if shards is None:
            shards = [torch.zeros(1 << self.n_local, dtype=dtype, device="cuda") for _ in range(1 << self.g)]
        if len(shards) != 1 << self.g:
            raise ValueError("need 2^global_bits shards")
        for t in shards:
            _check_state(t, "shard")
            if t.numel() != 1 << self.n_local or t.dtype != dtype:
                raise ValueError("every shard holds 2^(n - global_bits) amplitudes of the state's dtype")
        self.shards = list(shards)
        self.map = list(range(self.n))

    @classmethod
    def from_full(cls, psi: torch.Tensor, global_bits: int) -> "ShardedState":
        n = _nq(psi)
        parts = [c.clone() for c in psi.reshape(1 << global_bits, -1)]
        return cls(n, global_bits, psi.dtype, parts)

    def simulate(self, gates, theta=None, restore: bool = True, stream=None) -> "ShardedState":
        if self.map != list(range(self.n)):
            raise ValueError("the state's qubits are remapped; run from the identity map")
        arr, keep = _gate_array(gates)
        th = None if theta is None else np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        fmap = (ctypes.c_int32 * self.n)()
        check(lib().diaq_sharded_simulate(arr, len(gates), _dptr(th) if th is not None else None, self.n, self.g,
                                          _dtype_code(self.dtype), _shard_ptrs(self.shards), int(bool(restore)), fmap,
                                          _stream(stream)))
        self.map = list(fmap)
        return self

    def norm(self, stream=None) -> float:
        out = ctypes.c_double(0)
        check(lib().diaq_sharded_norm(_shard_ptrs(self.shards), self.n, self.g, _dtype_code(self.dtype),
                                      ctypes.byref(out), _stream(stream)))
        return out.value

    def expect(self, xmask, zmask, coeff, stream=None) -> complex:
        xm, zm, cc = _terms(xmask, zmask, coeff)
        m = (ctypes.c_int32 * self.n)(*self.map)
        out = np.zeros(2)
        check(lib().diaq_sharded_expect(_shard_ptrs(self.shards), self.n, self.g, _dtype_code(self.dtype), m, len(xm),
                                        xm.ctypes.data_as(N._u64p), zm.ctypes.data_as(N._u64p), _dptr(cc), _dptr(out),
                                        _stream(stream)))
        return complex(out[0], out[1])

    def physical(self) -> torch.Tensor:
        """The shards concatenated in shard order (physical index order)."""
        return torch.cat(self.shards)


class TorchDistTransport:
    """Pairwise buffer exchange between ranks with torch.distributed
    (NCCL for CUDA tensors, gloo for CPU tensors): send `send` to `partner`
    and receive its buffer into `recv`."""

    def exchange(self, partner: int, send: torch.Tensor, recv: torch.Tensor) -> None:
        import torch.distributed as dist
        ops = [dist.P2POp(dist.isend, send, partner), dist.P2POp(dist.irecv, recv, partner)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()


class ShardRank:
    """One rank's shard of a state over 2^global_bits ranks (rank r holds
    shard r) and its steps of diaq_shard_schedule: gates run on the shard in
    place; an exchange packs the half this rank gives away
    (diaq_shard_pack), trades buffers with the partner through a transport,
    and unpacks what it received (diaq_shard_unpack)."""

    def __init__(self, rank: int, n_qubits: int, global_bits: int, shard: torch.Tensor):
        self.rank, self.n, self.g = int(rank), int(n_qubits), int(global_bits)
        self.n_local = self.n - self.g
        _check_state(shard, "shard")
        if shard.numel() != 1 << self.n_local:
            raise ValueError("the shard holds 2^(n - global_bits) amplitudes")
        self.shard = shard
        self.send = torch.empty(1 << (self.n_local - 1), dtype=shard.dtype, device=shard.device)
        self.recv = torch.empty_like(self.send)
        self._ops = {}

    def plan(self, gates, theta=None, restore: bool = True) -> list:
        steps, self.final_map = shard_schedule(gates, self.n, self.g, restore)
        swap = _SwapGate()
        self._ops = {}
        for i, s in enumerate(steps):
            if s["kind"] == "exchange":
                continue
            g = gates[s["gate"]] if s["kind"] == "apply" else swap
            self._ops[i] = build(_Retargeted(g, s["targets"]), self.n_local, dtype=self.shard.dtype, theta=theta)
        return steps

    def apply_step(self, i: int, step: dict) -> None:
        apply(self._ops[i], self.shard, self.shard)

    def partner(self, step: dict) -> int:
        return self.rank ^ (1 << step["global_bit"])

    def _value(self, step: dict) -> int:
        return 1 - ((self.rank >> step["global_bit"]) & 1)

    def pack(self, step: dict, stream=None) -> torch.Tensor:
        check(lib().diaq_shard_pack(ctypes.c_void_p(self.shard.data_ptr()), self.n_local, _dtype_code(self.shard.dtype),
                                    step["local_bit"], self._value(step), ctypes.c_void_p(self.send.data_ptr()),
                                    _stream(stream)))
        return self.send

    def unpack(self, step: dict, stream=None) -> None:
        check(lib().diaq_shard_unpack(ctypes.c_void_p(self.recv.data_ptr()), ctypes.c_void_p(self.shard.data_ptr()),
                                      self.n_local, _dtype_code(self.shard.dtype), step["local_bit"],
                                      self._value(step), _stream(stream)))

    def run(self, gates, theta=None, restore: bool = True, transport=None) -> list:
        """All steps on this rank; the other ranks run the same call."""
        transport = transport or TorchDistTransport()
        steps = self.plan(gates, theta, restore)
        for i, s in enumerate(steps):
            if s["kind"] == "exchange":
                self.pack(s)
                torch.cuda.current_stream().synchronize()
                transport.exchange(self.partner(s), self.send, self.recv)
                self.unpack(s)
            else:
                self.apply_step(i, s)
        return self.final_map


class _Retargeted:
    """A gate object with its targets replaced (same matrix or generator)."""

    def __init__(self, g, targets):
        self.targets = tuple(targets)
        self.matrix = getattr(g, "matrix", None)
        self.param = int(getattr(g, "param", -1))
        self.gen = getattr(g, "gen", "")
        self.scale = float(getattr(g, "scale", 1.0))


class _SwapGate:
    targets = (1, 0)
    matrix = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
    param = -1
    gen = ""
    scale = 1.0
