"""Failure detection without a GPU fault: a device wait that nothing
completes gives up after its time limit and the host reads the status; the
context stays usable."""
import time

import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    w = synth.Workload("fail", 16, 4, 20, tau=4.0, seed=1)
    F = synth.blocks(w)
    with btt.Operator(F, precision="bf16", gemm="tensor", max_nrhs=16) as op:
        lib = btt.load()
        st = torch.cuda.current_stream().cuda_stream
        t0 = time.perf_counter()
        rc = lib.btt_selftest_wait(op.handle, 0.2, st)
        dt = time.perf_counter() - t0
        assert rc == _lib.BTT_ERR_TIMEOUT, lib.btt_last_error()
        assert 0.2 <= dt < 5.0
        assert b"bounded" in lib.btt_last_error()
        op.device_status()                       # the code was cleared
        m = synth.vectors(w, "m", 16).astype(np.float32)
        y = op.matvec(torch.from_numpy(m).cuda())
        op.device_status()
        assert direct.rel_l2(y.double().cpu().numpy(), direct.forward(F, m.astype(np.float64))) < 1e-2
