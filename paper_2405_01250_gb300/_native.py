"""ctypes declarations of the C ABI in include/diaq.h (libdiaq_gb300.so).

The library is loaded from this package's _build/ directory. There is no
fallback: if it is missing, every entry point raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# DIAQ_DEBUG_BOUNDS=1 selects the debug build, whose kernels check every
# computed index (diaq_debug_bounds_check reports a failure)
DEBUG_BOUNDS = os.environ.get("DIAQ_DEBUG_BOUNDS", "0") == "1"
LIB_PATH = os.path.join(HERE, "_build_dbg" if DEBUG_BOUNDS else "_build",
                        "libdiaq_gb300_dbg.so" if DEBUG_BOUNDS else "libdiaq_gb300.so")

DIAQ_MAX_K = 6
DIAQ_MAX_QUBITS = 34

STATUS = {
    0: "DIAQ_OK", 1: "DIAQ_ERR_ARG", 2: "DIAQ_ERR_SHAPE", 3: "DIAQ_ERR_ALLOC", 4: "DIAQ_ERR_CUDA",
    5: "DIAQ_ERR_TIMEOUT", 6: "DIAQ_ERR_BOUNDS", 7: "DIAQ_ERR_UNSUPPORTED",
}
C64, C128 = 0, 1
ONTHEFLY, STORED = 0, 1
CLASSES = {0: "general", 1: "real", 2: "diagonal", 3: "permutation", 4: "monomial", 5: "raw"}


class DiaqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class diaq_gate(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32),
        ("targets", ctypes.c_int32 * DIAQ_MAX_K),
        ("m", ctypes.POINTER(ctypes.c_double)),
        ("param", ctypes.c_int32),
        ("scale", ctypes.c_double),
        ("gen", ctypes.c_char * (DIAQ_MAX_K + 2)),
    ]


class diaq_op_info(ctypes.Structure):
    _fields_ = [
        ("n_qubits", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("op_class", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("targets", ctypes.c_int32 * DIAQ_MAX_K),
        ("n_diagonals", ctypes.c_int64),
        ("stored_bytes", ctypes.c_int64),
        ("real_values", ctypes.c_int32),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p
_op = ctypes.c_void_p
_gp = ctypes.POINTER(diaq_gate)

# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "diaq_last_error": (ctypes.c_char_p, []),
    "diaq_version": (ctypes.c_char_p, []),
    "diaq_gate_offsets": (ctypes.c_int, [_gp, ctypes.c_int32, _i64p, ctypes.c_int64, _i64p]),
    "diaq_diaq_matmul_host": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _i64p, _dp, ctypes.c_int64, _i64p, _dp,
                                             _i64p, _i64p, _i64p, _dp]),
    "diaq_fuse_gates_host": (ctypes.c_int, [_gp, ctypes.c_int32, _dp, _i32p, _i32p, _dp]),
    "diaq_build": (ctypes.c_int, [_gp, ctypes.c_int32, ctypes.c_int, ctypes.c_int, _dp, _vp,
                                  ctypes.POINTER(_op)]),
    "diaq_build_diaq": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _i64p, _dp, ctypes.c_int, _vp,
                                       ctypes.POINTER(_op)]),
    "diaq_op_destroy": (ctypes.c_int, [_op]),
    "diaq_op_query": (ctypes.c_int, [_op, ctypes.POINTER(diaq_op_info)]),
    "diaq_op_offsets": (ctypes.c_int, [_op, _i64p, ctypes.c_int64, _i64p]),
    "diaq_op_read_diagonal": (ctypes.c_int, [_op, ctypes.c_int64, _vp, _vp]),
    "diaq_fuse": (ctypes.c_int, [ctypes.POINTER(_op), ctypes.c_int32, ctypes.c_int, _vp, ctypes.POINTER(_op)]),
    "diaq_apply": (ctypes.c_int, [_op, _vp, _vp, _vp]),
    "diaq_op_apply_bytes": (ctypes.c_int, [_op, ctypes.c_int32, _i64p]),
    "diaq_op_diagonal_nnz": (ctypes.c_int, [_op, _i64p, _vp]),
    "diaq_op_prune": (ctypes.c_int, [_op, _vp, ctypes.POINTER(_op)]),
    "diaq_unitary_chain": (ctypes.c_int, [_gp, ctypes.c_int32, _dp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                                          _i64p, _i64p, _vp, ctypes.POINTER(_op)]),
    "diaq_simulate": (ctypes.c_int, [ctypes.POINTER(_op), ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "diaq_simulate_bytes": (ctypes.c_int, [ctypes.POINTER(_op), ctypes.c_int32, _i64p]),
    "diaq_simulate_timed": (ctypes.c_int, [ctypes.POINTER(_op), ctypes.c_int32, _vp, _vp, _vp, _vp, _vp,
                                           ctypes.POINTER(ctypes.c_float)]),
    "diaq_norm": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int, _dp, _vp]),
    "diaq_expect": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, _u64p, _u64p, _dp, _dp, _vp]),
    "diaq_apply_pauli_sum": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, _u64p, _u64p,
                                            _dp, _vp]),
    "diaq_adjoint_grad": (ctypes.c_int, [_gp, ctypes.c_int32, _dp, ctypes.c_int32, ctypes.c_int32, _u64p, _u64p,
                                         _dp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int, _dp, _dp, _vp]),
    "diaq_sample": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int, _vp, ctypes.c_int64, _vp, _vp]),
    "diaq_norm_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int, _dp, _vp]),
    "diaq_debug_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int32]),
    "diaq_debug_bounds_enabled": (ctypes.c_int, [_i32p]),
    "diaq_debug_bounds_check": (ctypes.c_int, [ctypes.c_int32, _u64p]),
    "diaq_debug_bounds_status": (ctypes.c_int, [ctypes.c_uint64]),
}

class diaq_batch_tuning(ctypes.Structure):
    _fields_ = [
        ("n_tried", ctypes.c_int32),
        ("cluster", ctypes.c_int32 * 24),
        ("threads", ctypes.c_int32 * 24),
        ("window", ctypes.c_int32 * 24),
        ("lanes", ctypes.c_int32 * 24),
        ("ms", ctypes.c_float * 24),
        ("best_cluster", ctypes.c_int32),
        ("best_threads", ctypes.c_int32),
        ("best_window", ctypes.c_int32),
        ("best_lanes", ctypes.c_int32),
        ("best_ms", ctypes.c_float),
    ]


class diaq_apply_tuning(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int32),
        ("k", ctypes.c_int32 * 27),
        ("threads", ctypes.c_int32 * 27),
        ("groups", ctypes.c_int32 * 27),
        ("ms", ctypes.c_float * 27),
        ("best_threads", ctypes.c_int32 * 3),
        ("best_groups", ctypes.c_int32 * 3),
        ("best_ms", ctypes.c_float * 3),
    ]


class diaq_plan_tuning(ctypes.Structure):
    _fields_ = [
        ("n_tried", ctypes.c_int32),
        ("window", ctypes.c_int32 * 12),
        ("lanes", ctypes.c_int32 * 12),
        ("blocks", ctypes.c_int32 * 12),
        ("ms", ctypes.c_float * 12),
        ("best_window", ctypes.c_int32),
        ("best_lanes", ctypes.c_int32),
        ("best_blocks", ctypes.c_int32),
        ("best_ms", ctypes.c_float),
    ]


class diaq_fusion_tuning(ctypes.Structure):
    _fields_ = [
        ("n_depths", ctypes.c_int32),
        ("ops", ctypes.c_int32 * 8),
        ("ms", ctypes.c_float * 8),
        ("best_depth", ctypes.c_int32),
    ]


SIGNATURES.update({
    "diaq_autotune_apply": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int, _vp, _vp, ctypes.c_int32,
                                           ctypes.POINTER(diaq_apply_tuning), _vp]),
    "diaq_set_apply_launch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "diaq_plan_fusion": (ctypes.c_int, [_gp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p]),
    "diaq_plan_fusion_commuting": (ctypes.c_int, [_gp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                                  _i32p]),
    "diaq_plan_fusion_diagonal": (ctypes.c_int, [_gp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p]),
    "diaq_autotune_fusion": (ctypes.c_int, [_gp, ctypes.c_int32, _dp, ctypes.c_int32, ctypes.c_int, _vp,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(diaq_fusion_tuning), _vp]),
    "diaq_adjoint_plan_create": (ctypes.c_int, [_gp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _u64p, _u64p,
                                                _dp, ctypes.c_int32, ctypes.c_int, ctypes.POINTER(_vp)]),
    "diaq_adjoint_plan_run": (ctypes.c_int, [_vp, _dp, _vp, _dp, _dp, _vp]),
    "diaq_adjoint_plan_destroy": (ctypes.c_int, [_vp]),
    "diaq_adjoint_plan_set_window": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_adjoint_plan_set_sweep": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "diaq_adjoint_plan_get_sweep": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "diaq_adjoint_plan_autotune": (ctypes.c_int, [_vp, _dp, ctypes.c_int32, ctypes.POINTER(diaq_plan_tuning)]),
    "diaq_adjoint_plan_set_blocks": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_adjoint_plan_get_blocks": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "diaq_batch_set_window": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_batch_get_window": (ctypes.c_int, [_vp, _i32p]),
    "diaq_batch_set_sweep": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "diaq_batch_get_sweep": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "diaq_batch_set_runs": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_batch_get_runs": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "diaq_adjoint_plan_get_window": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "diaq_adjoint_plan_set_runs": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_adjoint_plan_get_runs": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "diaq_adjoint_plan_set_scaled": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_adjoint_plan_set_pairs": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_adjoint_plan_get_pairs": (ctypes.c_int, [_vp, _i32p]),
    "diaq_adjoint_plan_get_scaled": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "diaq_batch_set_scaled": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "diaq_batch_get_scaled": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "diaq_batch_create": (ctypes.c_int, [ctypes.c_int32, _i32p, _i32p, _gp, _i32p, _i32p, _u64p, _u64p, _dp,
                                         ctypes.c_int, ctypes.POINTER(_vp)]),
    "diaq_batch_destroy": (ctypes.c_int, [_vp]),
    "diaq_batch_set_launch": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "diaq_batch_run": (ctypes.c_int, [_vp, _dp, _dp, _dp, _vp]),
    "diaq_batch_autotune": (ctypes.c_int, [_vp, _dp, ctypes.c_int32, ctypes.POINTER(diaq_batch_tuning), _vp]),
    "diaq_batch_query": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p, _i64p]),
})

class diaq_shard_step(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("gate", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("targets", ctypes.c_int32 * DIAQ_MAX_K),
        ("global_bit", ctypes.c_int32),
        ("local_bit", ctypes.c_int32),
    ]


SHARD_APPLY, SHARD_EXCHANGE, SHARD_LOCAL_SWAP = 0, 1, 2

SIGNATURES.update({
    "diaq_shard_schedule": (ctypes.c_int, [_gp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(diaq_shard_step), ctypes.c_int32, _i32p, _i32p]),
    "diaq_shard_swap": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, _vp]),
    "diaq_shard_pack": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
    "diaq_shard_unpack": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                         _vp]),
    "diaq_sharded_simulate": (ctypes.c_int, [_gp, ctypes.c_int32, _dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                             ctypes.POINTER(_vp), ctypes.c_int32, _i32p, _vp]),
    "diaq_sharded_norm": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int32, ctypes.c_int, _dp,
                                         _vp]),
    "diaq_sharded_expect": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int32, ctypes.c_int, _i32p,
                                           ctypes.c_int32, _u64p, _u64p, _dp, _dp, _vp]),
})

_LIB = None


def lib() -> ctypes.CDLL:
    """Load libdiaq_gb300.so (after torch, so both share one CUDA runtime)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libdiaq_gb300.so is not built ({LIB_PATH} missing); run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        try:
            import torch  # noqa: F401  (loads libcudart first)
        except ImportError:
            pass
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status: int) -> None:
    if status != 0:
        msg = lib().diaq_last_error().decode(errors="replace")
        raise DiaqError(status, msg)
