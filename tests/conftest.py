import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(autouse=True)
def _checked_build_report(request):
    """Under the checked build (PAB_CHECKED=1), every GPU test ends with the library's bounds
    report: any index a kernel met outside its buffer fails the test that launched it."""
    yield
    if "gpu" not in request.keywords or os.environ.get("PAB_CHECKED", "") != "1":
        return
    from paper_2511_21031_gb300 import pab
    rep = pab.pab_check_report()
    assert rep is not None, "PAB_CHECKED=1 but the loaded library is not the checked build"
    assert rep["count"] == 0, f"out-of-bounds index in the kernels: {rep}"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device in this process")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
