import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running case")


import pytest  # noqa: E402


@pytest.fixture(autouse=True)
def _debug_bounds_clean(request):
    """With DIAQ_DEBUG_BOUNDS=1 (the library's index-checking debug build),
    every GPU test must leave no failed device index check behind."""
    yield
    if os.environ.get("DIAQ_DEBUG_BOUNDS", "0") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import ctypes

    import torch
    from paper_2405_01250_gb300 import _native
    torch.cuda.synchronize()
    word = ctypes.c_uint64(0)
    st = _native.lib().diaq_debug_bounds_check(1, ctypes.byref(word))
    assert st == 0, _native.lib().diaq_last_error().decode()
