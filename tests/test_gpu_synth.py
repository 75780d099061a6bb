"""The device build of the input generator against the host build: the GPU
runs fill whole tensors on the device, the oracle draws entries on the host,
so both must give the same numbers (to the rounding of their transcendental
functions)."""
import numpy as np
import pytest
import torch

import synth
from synth import philox

pytestmark = pytest.mark.gpu


def _dev():
    return synth.dev_lib()


def test_normal_and_uniform_match_host():
    n, start = 100_003, 77
    out64 = torch.empty(n, dtype=torch.float64, device="cuda")
    out32 = torch.empty(n, dtype=torch.float32, device="cuda")
    # one output per call: FP64 when given, else FP32
    assert _dev().synth_dev_normal(5, synth.workloads.T_PARAM, start, n, out64.data_ptr(), None, None) == 0
    assert _dev().synth_dev_normal(5, synth.workloads.T_PARAM, start, n, None, out32.data_ptr(), None) == 0
    torch.cuda.synchronize()
    ref = synth.normals(5, synth.workloads.T_PARAM, n, start=start)
    np.testing.assert_allclose(out64.cpu().numpy(), ref, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(out32.cpu().numpy(), ref.astype(np.float32), rtol=2e-7, atol=1e-7)
    # the numpy build too, on a slice
    np.testing.assert_allclose(ref[:1000], philox.normal(5, synth.workloads.T_PARAM,
                                                         np.arange(start, start + 1000, dtype=np.uint64)),
                               rtol=1e-13, atol=1e-14)

    u = torch.empty(n, dtype=torch.float64, device="cuda")
    assert _dev().synth_dev_uniform(9, synth.workloads.T_NOISE, 0, n, 0.5, 2.0, u.data_ptr(), None, None) == 0
    torch.cuda.synchronize()
    uref = synth.uniforms(9, synth.workloads.T_NOISE, n, 0.5, 2.0)
    np.testing.assert_allclose(u.cpu().numpy(), uref, rtol=1e-15, atol=0)
    assert float(u.min()) >= 0.5 and float(u.max()) <= 2.0


@pytest.mark.parametrize("envelope", [False, True])
def test_blocks_match_host(envelope):
    w = synth.Workload("gen", 37, 13, 211, tau=9.0, envelope=envelope, seed=4)
    k0, k1 = 3, 29
    ed, em = synth.workloads.envelope(w, "d"), synth.workloads.envelope(w, "m")
    ed_t = None if ed is None else torch.from_numpy(ed).cuda()
    em_t = None if em is None else torch.from_numpy(em).cuda()
    out = torch.empty((k1 - k0, w.N_d, w.N_m), dtype=torch.float64, device="cuda")
    rc = _dev().synth_dev_blocks(w.seed, w.N_d, w.N_m, float(w.tau),
                                 None if ed_t is None else ed_t.data_ptr(),
                                 None if em_t is None else em_t.data_ptr(),
                                 k0, k1, out.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    ref = synth.blocks(w, k0, k1)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-15)
