import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a B300 GPU and the built CUDA library")


def pytest_collection_modifyitems(config, items):
    # GPU tests run only where CUDA is present; the CPU suite never touches the device.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _bounds_checked_build(request):
    """Under SDG_EXPECT_CHECKED=1 (the bounds-checked run of the GPU suite, tests/test_gpu_checked.py) every GPU
    test must run on libsdg_checked.so and leave its out-of-range status word at 0."""
    yield
    if os.environ.get("SDG_EXPECT_CHECKED") != "1" or "gpu" not in request.keywords:
        return
    import paper_2305_13220_b300 as sdg
    status, checked = sdg._abi.checked_status(0, clear=True)
    assert checked, "SDG_EXPECT_CHECKED=1 but the loaded library is not the bounds-checked build"
    assert status == 0, f"bounds-checked build recorded an index out of range: code {status >> 48}, " \
                        f"index {status & 0xFFFFFFFFFFFF}"
