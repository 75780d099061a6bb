"""Edge cases of the cluster time transforms (four CTAs per transform tile,
sub-blocks exchanged through distributed shared memory) against the FP64
oracle.

On the long fixed plans the input transforms (complex64 and the BF16
tensor-core operand form) run on clusters whose tile is four CTAs' columns
wide at 2 N_t in {2000, 2048, 4000, 4096, 8000}, the complex64 inverse at
{2048, 4000, 4096, 8000} and the BF16 inverse at {4000, 4096, 8000}; the
other inverse forms at these lengths keep one-CTA tiles.  These cases give
them column counts below one cluster tile, ragged last tiles, several
tiles, several vectors, and vectors at odd addresses through pointer
tables.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from tests.test_gpu_parity import TOL, dev, host, inputs
from tests.test_gpu_quad import _batched

pytestmark = pytest.mark.gpu

# (N_t, N_d, N_m): 2 N_t = 2000 (tile 32 columns), 2048 (32), 4000 (16),
# 4096 (16), 8000 (8); N_m below, at and above one tile, ragged
SHAPES = [(1000, 3, 37), (1000, 5, 130), (1000, 1, 5), (1024, 3, 45), (2000, 2, 21),
          (2048, 2, 19), (4000, 1, 9)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_cluster_transforms(shape):
    N_t, N_d, N_m = shape
    w = synth.Workload("clus", N_t, N_d, N_m, tau=N_t / 4, seed=N_m + 13 * N_d)
    F, m, d, g = inputs(w, nrhs=2)
    with btt.Operator(torch.from_numpy(F).cuda(), precision="f32", max_nrhs=2) as op:
        dm = host(op.matvec(dev(m, torch.float32)))
        md = host(op.adjoint(dev(d, torch.float32)))
        hm = host(op.hessian(dev(m, torch.float32), dev(g, torch.float32)))
        op.device_status()
    assert direct.rel_l2(dm, direct.forward(F, m)) < TOL["f32"]
    assert direct.rel_l2(md, direct.adjoint(F, d)) < TOL["f32"]
    assert direct.rel_l2(hm, direct.hessian(F, m, g)) < TOL["f32"]


@pytest.mark.parametrize("N_t", [1000, 2000])
def test_cluster_pointer_tables_at_odd_addresses(N_t):
    """Vectors 4 bytes past a 16-byte boundary through btt_hessian_batched
    give results bit-identical to the contiguous batch."""
    N_d, N_m, nrhs = 3, 70, 3
    w = synth.Workload("clusptr", N_t, N_d, N_m, tau=N_t / 4, seed=N_t + 5)
    F, m, _, g = inputs(w, nrhs=nrhs)
    n = N_t * N_m
    with btt.Operator(torch.from_numpy(F).cuda(), precision="f32", max_nrhs=nrhs) as op:
        gt = dev(g, torch.float32)
        ref = host(op.hessian(dev(m, torch.float32), gt))
        pool = torch.zeros(nrhs * (n + 4) + 4, dtype=torch.float32, device="cuda")
        outp = torch.zeros_like(pool)
        xs = [pool[1 + b * (n + 4): 1 + b * (n + 4) + n] for b in range(nrhs)]
        ys = [outp[3 + b * (n + 4): 3 + b * (n + 4) + n] for b in range(nrhs)]
        for b in range(nrhs):
            xs[b].copy_(torch.from_numpy(m[b].astype(np.float32).ravel()))
        _batched(op, xs, gt, ys)
        got = np.stack([y.double().cpu().numpy().reshape(N_t, N_m) for y in ys])
        op.device_status()
    np.testing.assert_array_equal(got, ref)
    assert direct.rel_l2(got, direct.hessian(F, m, g)) < TOL["f32"]


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
@pytest.mark.parametrize("shape", [(1000, 5, 37), (1024, 9, 70), (2000, 3, 21), (2048, 2, 9)])
def test_tensor_cluster_transforms(shape, prec):
    """The BF16 tensor-core operand transform (conj spectra as BF16 pairs,
    and the remainder plane of the split pair) and the BF16 inverse on
    cluster tiles."""
    N_t, N_d, N_m = shape
    w = synth.Workload("clustc", N_t, N_d, N_m, tau=N_t / 4, seed=N_m + 17 * N_d)
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
