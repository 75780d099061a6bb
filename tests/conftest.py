import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(autouse=True)
def _bounds_check_record(request):
    """Under the bounds-check build (BTT_CHECK=1) every GPU test must leave no
    recorded out-of-range index behind."""
    yield
    if request.node.get_closest_marker("gpu") is None or os.environ.get("BTT_CHECK", "0") in ("", "0"):
        return
    from paper_2407_13066_gb300 import _lib
    lib = _lib.load()
    st = lib.btt_check_status(None)
    assert st == _lib.BTT_OK, lib.btt_last_error().decode()
