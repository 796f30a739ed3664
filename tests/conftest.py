import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libhj.so")


def pytest_collection_modifyitems(config, items):
    # without a GPU, gpu-marked tests are skipped rather than failed when they are selected
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _debug_build_checks(request):
    """With the debug library (HJ_LIBRARY=debug), every GPU test ends with the
    library's memory checks: no index out of range in a kernel, no guard band
    of a device allocation overwritten."""
    yield
    if os.environ.get("HJ_LIBRARY") != "debug" or "gpu" not in request.keywords:
        return
    import paper_2006_16465_gb300 as hj
    code, site, index = hj.hj_debug_check()
    assert code == hj.HJ_OK, f"debug check after {request.node.name}: site {site}, index {index}"
