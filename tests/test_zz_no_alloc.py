"""diaq_norm_noalloc: the norm for callers that cannot allocate device memory
(an application whose memory manager owns the whole device heap, or a
latency-critical loop that must not pay for allocation). It keeps its
partial sums in a fixed array inside the library; this checks, through the
C ABI, that it returns what diaq_norm returns, on consecutive calls that
reuse the array with different sizes and precisions.

Collected last on purpose (file name), so a run that stops at the first
failure has run every other test before it."""

import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import _native
    return _native.lib()


def _norm(lib, fn, t, n, code):
    out = ctypes.c_double(0)
    st = getattr(lib, fn)(ctypes.c_void_p(t.data_ptr()), n, code, ctypes.byref(out),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.diaq_last_error().decode()
    return out.value


def test_norm_noalloc_matches_norm_on_consecutive_calls(lib):
    rng = np.random.default_rng(11)
    # large then small then large again: a later call must not see the
    # earlier call's partial sums left in the shared array
    cases = [(22, torch.complex128), (9, torch.complex128), (17, torch.complex64), (3, torch.complex64),
             (20, torch.complex128)]
    for n, dt in cases:
        psi = torch.as_tensor(synth.random_state(n, rng) * 1.3).to(device="cuda", dtype=dt)
        code = 1 if dt == torch.complex128 else 0
        ref = _norm(lib, "diaq_norm", psi, n, code)
        first = _norm(lib, "diaq_norm_noalloc", psi, n, code)
        second = _norm(lib, "diaq_norm_noalloc", psi, n, code)
        tol = (1e-13 if dt == torch.complex128 else 1e-6) * ref
        assert abs(first - ref) <= tol, (n, dt, first, ref)
        assert abs(second - ref) <= tol, (n, dt, second, ref)


def test_norm_noalloc_rejects_bad_arguments(lib):
    out = ctypes.c_double(0)
    assert lib.diaq_norm_noalloc(None, 4, 1, ctypes.byref(out), None) == 1
    assert b"NULL" in lib.diaq_last_error()
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    assert lib.diaq_norm_noalloc(ctypes.c_void_p(t.data_ptr()), 0, 1, ctypes.byref(out), None) == 1
