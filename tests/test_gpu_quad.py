"""Edge cases of the quad time transforms (paired FP32 lanes, four real
columns per butterfly) against the FP64 oracle.

The quad kernels run for 2 N_t in {256, 512, 1024} (inverse transforms;
the BF16 tensor-core inverse also at 2048) and {512, 1024} (the BF16
tensor-core input transform).  These cases give them column counts that
leave a partial quad (N_m and N_d not multiples of 4), rows that are not
16-byte aligned, vectors passed through pointer tables at odd addresses, and
the CG step fused into the inverse transform.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import _lib
from tests.test_gpu_cg import system
from tests.test_gpu_parity import TOL, dev, host, inputs

pytestmark = pytest.mark.gpu

# (N_t, N_d, N_m): N_m = 4k + 1, 4k + 2, 4k + 3 and N_d odd, so both the
# parameter-side and the data-side transforms end in a partial quad
RAGGED = [(128, 3, 37), (128, 5, 42), (256, 7, 67), (256, 1, 5), (512, 3, 45), (1024, 5, 30)]


@pytest.mark.parametrize("shape", RAGGED)
def test_fp32_ragged_quads(shape):
    N_t, N_d, N_m = shape
    w = synth.Workload("quad", N_t, N_d, N_m, tau=N_t / 4, seed=N_m + 7 * N_d)
    F, m, d, g = inputs(w, nrhs=2)
    with btt.Operator(torch.from_numpy(F).cuda(), precision="f32", max_nrhs=2) as op:
        dm = host(op.matvec(dev(m, torch.float32)))
        md = host(op.adjoint(dev(d, torch.float32)))
        hm = host(op.hessian(dev(m, torch.float32), dev(g, torch.float32)))
    assert direct.rel_l2(dm, direct.forward(F, m)) < TOL["f32"]
    assert direct.rel_l2(md, direct.adjoint(F, d)) < TOL["f32"]
    assert direct.rel_l2(hm, direct.hessian(F, m, g)) < TOL["f32"]


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
@pytest.mark.parametrize("shape", [(128, 9, 37), (256, 17, 66), (512, 5, 43), (1024, 3, 21)])
def test_tensor_ragged_quads(shape, prec):
    N_t, N_d, N_m = shape
    w = synth.Workload("quadtc", N_t, N_d, N_m, tau=N_t / 4, seed=N_m + 11 * N_d)
    F, m, d, g = inputs(w, nrhs=16)
    with btt.Operator(torch.from_numpy(F).cuda(), precision=prec, max_nrhs=16, gemm="tensor") as op:
        dm = host(op.matvec(dev(m, torch.float32)))
        md = host(op.adjoint(dev(d, torch.float32)))
        hm = host(op.hessian(dev(m, torch.float32), dev(g, torch.float32)))
        op.device_status()
    tol = TOL[prec]
    assert direct.rel_l2(dm, direct.forward(F, m)) < tol
    assert direct.rel_l2(md, direct.adjoint(F, d)) < tol
    assert direct.rel_l2(hm, direct.hessian(F, m, g)) < 2 * tol


def _batched(op, xs, g, ys):
    lib = _lib.load()
    mp = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.btt_hessian_batched(op.handle, mp, g.data_ptr(), yp, len(xs), st))
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec,gemm", [("f32", "simt"), ("bf16", "tensor"), ("bf16x2", "tensor")])
@pytest.mark.parametrize("N_t", [64, 128, 256, 512, 1024])
def test_pointer_tables_at_odd_addresses(N_t, prec, gemm):
    """Vectors at addresses 4 bytes past a 16-byte boundary (rows not
    16-byte aligned: the quad and one-exchange kernels take their
    element-wise loads and stores) give results bit-identical to the
    contiguous batch, at every one-exchange length (2 N_t = 128 .. 2048)."""
    N_d, N_m, nrhs = 6, 48, 16
    w = synth.Workload("quadptr", N_t, N_d, N_m, tau=N_t / 4, seed=N_t + 1)
    F, m, _, g = inputs(w, nrhs=nrhs)
    n = N_t * N_m
    with btt.Operator(torch.from_numpy(F).cuda(), precision=prec, max_nrhs=nrhs, gemm=gemm) as op:
        gt = dev(g, torch.float32)
        ref = host(op.hessian(dev(m, torch.float32), gt))
        pool = torch.zeros(nrhs * (n + 4) + 4, dtype=torch.float32, device="cuda")
        outp = torch.zeros_like(pool)
        xs = [pool[1 + b * (n + 4): 1 + b * (n + 4) + n] for b in range(nrhs)]
        ys = [outp[3 + b * (n + 4): 3 + b * (n + 4) + n] for b in range(nrhs)]
        for b in range(nrhs):
            xs[b].copy_(torch.from_numpy(m[b].astype(np.float32).ravel()))
        assert all(x.data_ptr() % 16 != 0 for x in xs) and all(y.data_ptr() % 16 != 0 for y in ys)
        _batched(op, xs, gt, ys)
        got = np.stack([y.double().cpu().numpy().reshape(N_t, N_m) for y in ys])
        op.device_status()
    np.testing.assert_array_equal(got, ref)
    assert direct.rel_l2(got, direct.hessian(F, m, g)) < 2 * TOL[prec]


@pytest.mark.parametrize("prec,gemm,tol,bound", [("f32", "simt", 1e-6, 2e-4), ("bf16", "tensor", 1e-3, 2e-2)])
def test_cg_fused_step_ragged_quads(prec, gemm, tol, bound):
    """CG with its step fused into the quad inverse transform (2 N_t = 256)
    on N_m = 10 columns (a partial last quad), against a dense solve."""
    w, F, g, H, lam = system(128, 3, 10, 21)
    alpha = lam / 50.0
    nrhs = 3
    b = synth.vectors(w, "m", nrhs).astype(np.float32)
    ref = np.stack([np.linalg.solve(H + alpha * np.eye(H.shape[0]), b[j].astype(np.float64).ravel())
                    for j in range(nrhs)]).reshape(b.shape)
    with btt.Operator(F, precision=prec, max_nrhs=nrhs, gemm=gemm) as op:
        x, its, rel = op.cg(torch.from_numpy(b).cuda(), alpha, gamma_inv=torch.from_numpy(g).cuda(),
                            tol=tol, max_iter=400)
        op.device_status()
    x = x.double().cpu().numpy()
    assert all(0 < i < 400 for i in its), its
    assert all(r <= tol for r in rel), rel
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    assert err < bound, err
