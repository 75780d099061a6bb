"""btt_matvec_noalloc: the F action for callers that cannot allocate.

A custom call inside another framework's execution step, a plugin limited
to a preallocated arena, or a real-time loop may not call cudaMalloc when it
applies the operator.  This entry point takes Fhat, m and d from the caller
and draws its scratch from a fixed device array inside the library.  The
test compares it, through the C ABI, with btt_matvec on the same operator
(and with the FP64 oracle) on two calls in a row, and checks that sizes
beyond the fixed scratch are refused with a clear message.  The file sorts
last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import _lib

pytestmark = pytest.mark.gpu


# (N_t, N_d, N_m): 2N_t = 250 runs the generic transforms; 2N_t = 128 the
# fixed-plan pair transforms and 2N_t = 2000 the cluster input transform,
# both of which read the quad twiddle copy and the position table that this
# entry point builds in its fixed scratch; 2N_t = 512, 1024 and 2048 the
# one-exchange transforms (stage 2 with a length-1, 2 and 4 step), which
# read the lane-pair twiddles it builds there (N_m odd: a ragged last tile)
SHAPES = [(125, 9, 61), (64, 8, 300), (1000, 10, 203), (256, 7, 301), (512, 6, 99), (1024, 5, 101)]


@pytest.mark.parametrize("shape", SHAPES, ids=["L250", "L128", "L2000", "L512", "L1024", "L2048"])
def test_noalloc_matches_matvec_on_two_calls(shape):
    lib = btt.load()
    N_t, N_d, N_m = shape
    w = synth.Workload("noalloc", N_t, N_d, N_m, tau=N_t / 4, seed=21)   # ragged N_m
    F = synth.blocks(w)
    with btt.Operator(F, precision="f32", max_nrhs=3) as op:
        raw, _ = op.copy_fhat()
        fhat = torch.from_numpy(raw).cuda()          # caller-owned copy of Fhat
        ms = [synth.vectors(w, "m", n, tensor_id=30 + n).astype(np.float32) for n in (1, 3)]
        m_dev = [torch.from_numpy(m).cuda() for m in ms]
        outs = [torch.full((m.shape[0], w.N_t, w.N_d), float("nan"), device="cuda") for m in ms]
        refs = [op.matvec(m) for m in m_dev]
        torch.cuda.synchronize()
        st = torch.cuda.current_stream().cuda_stream
        free_before = None
        for call, (m, out) in enumerate(zip(m_dev, outs)):
            if call == 1:
                free_before = torch.cuda.mem_get_info()[0]
            rc = lib.btt_matvec_noalloc(fhat.data_ptr(), w.N_t, w.N_d, w.N_m, m.data_ptr(),
                                        out.data_ptr(), m.shape[0], st)
            assert rc == _lib.BTT_OK, lib.btt_last_error()
            torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        for m, out, ref in zip(ms, outs, refs):
            got = out.double().cpu().numpy()
            assert direct.rel_l2(got, ref.double().cpu().numpy()) < 1e-5
            assert direct.rel_l2(got, direct.forward(F, m.astype(np.float64))) < 1e-5


def test_noalloc_refuses_sizes_beyond_its_scratch():
    lib = btt.load()
    x = torch.zeros(16, device="cuda")
    # the bandwidth operator's spectra need ~81 MB, more than the 32 MiB array
    rc = lib.btt_matvec_noalloc(x.data_ptr(), 1000, 100, 10000, x.data_ptr(), x.data_ptr(), 1, None)
    assert rc == _lib.BTT_ERR_UNSUPPORTED
    msg = lib.btt_last_error().decode()
    assert "scratch" in msg and "33554432" in msg
    assert lib.btt_matvec_noalloc(None, 4, 1, 1, x.data_ptr(), x.data_ptr(), 1, None) == _lib.BTT_ERR_ARG
    assert lib.btt_matvec_noalloc(x.data_ptr() + 4, 4, 1, 1, x.data_ptr(), x.data_ptr(), 1, None) == _lib.BTT_ERR_ARG
    # more vectors than one transform grid holds, refused before any launch
    rc = lib.btt_matvec_noalloc(x.data_ptr(), 1, 1, 1, x.data_ptr(), x.data_ptr(), 65536, None)
    assert rc == _lib.BTT_ERR_UNSUPPORTED and "nrhs" in lib.btt_last_error().decode()
    rc = lib.btt_matvec_noalloc(x.data_ptr(), 1, 1 << 16, 1 << 16, x.data_ptr(), x.data_ptr(), 1, None)
    assert rc == _lib.BTT_ERR_UNSUPPORTED
    torch.cuda.synchronize()
