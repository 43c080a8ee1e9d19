"""diaq_norm_noalloc: the norm for callers that cannot allocate device memory
(an application whose memory manager owns the whole device heap, or a
latency-critical loop that must not pay for allocation). It keeps its
partial sums in a fixed array inside the library. Checked through the C ABI:
it returns the same bits as diaq_norm and agrees with the FP64 oracle on
consecutive calls that reuse the array with different sizes and precisions,
and it makes no library allocation (an armed allocation-failure injection
is still armed after it).

Collected last on purpose (file name), so a run that stops at the first
failure has run every other test before it."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DIAQ_OK, DIAQ_ERR_ARG, DIAQ_ERR_ALLOC = 0, 1, 3


@pytest.fixture(scope="module")
def lib():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import _native
    return _native.lib()


def _call(lib, fn, t, n, code):
    out = ctypes.c_double(0)
    st = getattr(lib, fn)(ctypes.c_void_p(t.data_ptr()), n, code, ctypes.byref(out),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out.value


def _norm(lib, fn, t, n, code):
    st, v = _call(lib, fn, t, n, code)
    assert st == DIAQ_OK, lib.diaq_last_error().decode()
    return v


def test_norm_noalloc_matches_norm_on_consecutive_calls(lib):
    rng = np.random.default_rng(11)
    # large then small then large again: a later call must not see the
    # earlier call's partial sums left in the shared array
    cases = [(22, torch.complex128), (9, torch.complex128), (17, torch.complex64), (3, torch.complex64),
             (20, torch.complex128), (21, torch.complex64)]
    for n, dt in cases:
        psi = torch.as_tensor(synth.random_state(n, rng) * 1.3).to(device="cuda", dtype=dt)
        code = 1 if dt == torch.complex128 else 0
        ref = _norm(lib, "diaq_norm", psi, n, code)
        first = _norm(lib, "diaq_norm_noalloc", psi, n, code)
        second = _norm(lib, "diaq_norm_noalloc", psi, n, code)
        # the same kernels on the same grid: the same bits
        assert first == ref and second == ref, (n, dt, first, second, ref)
        # and the FP64 oracle's sum of |psi_i|^2 on the state as stored; the
        # complex64 path forms each square in FP32 (relative error 2^-24 per
        # term), the complex128 path differs only in summation order
        want = oracle.norm2(psi.cpu().numpy().astype(np.complex128))
        tol = (1e-13 if dt == torch.complex128 else 2.0 ** -22) * want
        assert abs(first - want) <= tol, (n, dt, first, want)


def test_norm_noalloc_makes_no_library_allocation(lib):
    """Arm the library's allocation-failure injection for its next
    allocation: diaq_norm_noalloc still succeeds and leaves it armed, so the
    following diaq_norm (which allocates its partials) fails with
    DIAQ_ERR_ALLOC. The injection acts on the host; no GPU work fails."""
    n = 18
    psi = torch.as_tensor(synth.random_state(n, np.random.default_rng(3))).to("cuda")
    ref = _norm(lib, "diaq_norm", psi, n, 1)
    assert lib.diaq_debug_inject_alloc_failure(0) == DIAQ_OK
    try:
        for _ in range(2):
            st, v = _call(lib, "diaq_norm_noalloc", psi, n, 1)
            assert st == DIAQ_OK, lib.diaq_last_error().decode()
            assert v == ref
        st, _ = _call(lib, "diaq_norm", psi, n, 1)
        assert st == DIAQ_ERR_ALLOC  # the injection was still armed
    finally:
        lib.diaq_debug_inject_alloc_failure(-1)
    assert _norm(lib, "diaq_norm", psi, n, 1) == ref


def test_norm_noalloc_rejects_bad_arguments(lib):
    out = ctypes.c_double(0)
    assert lib.diaq_norm_noalloc(None, 4, 1, ctypes.byref(out), None) == DIAQ_ERR_ARG
    assert b"NULL" in lib.diaq_last_error()
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    assert lib.diaq_norm_noalloc(ctypes.c_void_p(t.data_ptr()), 0, 1, ctypes.byref(out), None) == DIAQ_ERR_ARG
