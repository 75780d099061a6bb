"""The bounds-check build's reporting (BTT_CHECK=1 loads libbtt_check.so):
a kernel that tests an index beyond its extent, and skips the access, must
be reported once by btt_check_status and by btt_device_status, and the
record must then be clear.  In the normal build the self test is refused
and nothing is ever reported."""
import numpy as np
import pytest

import synth
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_check_record_reported_once():
    lib = btt.load()
    if lib.btt_check_build() != 1:
        assert lib.btt_check_selftest(None) == _lib.BTT_ERR_UNSUPPORTED
        assert lib.btt_check_status(None) == _lib.BTT_OK
        return
    assert lib.btt_check_status(None) == _lib.BTT_OK
    assert lib.btt_check_selftest(None) == _lib.BTT_OK
    assert lib.btt_check_status(None) == _lib.BTT_ERR_CUDA
    msg = lib.btt_last_error().decode()
    assert "selftest" in msg and "index 7" in msg
    assert lib.btt_check_status(None) == _lib.BTT_OK
    # an operator's device status reports the same record
    w = synth.Workload("chk", 16, 3, 5, tau=4.0, seed=2)
    with btt.Operator(synth.blocks(w), precision="f32") as op:
        assert lib.btt_check_selftest(None) == _lib.BTT_OK
        with pytest.raises(_lib.BttError, match="bounds check"):
            op.device_status()
        op.device_status()
