"""torch.autograd through the operator: backward of F is the hand-written F*
kernel.  Checked by central finite differences (step 1e-3, 8 random
directions) of a linear loss L(m) = <w, F m>, accumulated in FP64, and
against the oracle's transpose: on small FP32 operators, and on the
64-vector multi-right-hand-side workload through the tensor-core products
(BF16, BF16 hi+lo split pair) and the FP32 SIMT kernels."""
import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300.autograd import apply_F, apply_Fadj, apply_H

pytestmark = pytest.mark.gpu


def _setup(w, nrhs):
    F = synth.blocks(w)
    m = torch.from_numpy(synth.vectors(w, "m", nrhs).astype(np.float32)).cuda()
    wt = torch.from_numpy(synth.vectors(w, "d", nrhs, tensor_id=synth.workloads.T_WEIGHTS).astype(np.float32)).cuda()
    return F, m, wt


@pytest.mark.parametrize("shape", [(64, 8, 32), (256, 20, 500)])
def test_backward_is_adjoint_and_matches_finite_differences(shape):
    N_t, N_d, N_m = shape
    w = synth.Workload("ag", N_t, N_d, N_m, tau=N_t / 4, seed=17)
    F, m, wt = _setup(w, 2)
    op = btt.Operator(F, precision="f32", max_nrhs=2)
    x = m.clone().requires_grad_(True)
    loss = (apply_F(op, x).double() * wt.double()).sum()
    loss.backward()
    grad = x.grad.double().cpu().numpy()
    ref = direct.adjoint(F, wt.double().cpu().numpy())
    assert direct.rel_l2(grad, ref) < 1e-5

    def L(v):
        return float((op.matvec(v).double() * wt.double()).sum().cpu())

    h = 1e-3
    dirs = torch.from_numpy(synth.vectors(w, "m", 16, tensor_id=synth.workloads.T_DIRS)
                            .astype(np.float32)).cuda().reshape(8, 2, N_t, N_m)
    for v in dirs:
        fd = (L(m + h * v) - L(m - h * v)) / (2 * h)
        an = float((x.grad.double() * v.double()).sum().cpu())
        assert abs(fd - an) <= 1e-3 * abs(an) + 1e-6 * np.sqrt(m.numel()), (fd, an)
    op.close()


def test_adjoint_and_hessian_wrappers():
    w = synth.Workload("ag2", 50, 6, 40, tau=10.0, seed=3)
    F = synth.blocks(w)
    g = synth.noise_gamma_inv(w).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    op = btt.Operator(F, precision="f32")
    d = torch.from_numpy(synth.vectors(w, "d", 1)[0].astype(np.float32)).cuda().requires_grad_(True)
    wm = torch.from_numpy(synth.vectors(w, "m", 1, tensor_id=9)[0].astype(np.float32)).cuda()
    (apply_Fadj(op, d) * wm).sum().backward()
    assert direct.rel_l2(d.grad.double().cpu().numpy(), direct.forward(F, wm.double().cpu().numpy())) < 1e-5
    m = torch.from_numpy(synth.vectors(w, "m", 1)[0].astype(np.float32)).cuda().requires_grad_(True)
    (apply_H(op, m, gt) * wm).sum().backward()
    ref = direct.hessian(F, wm.double().cpu().numpy(), g.astype(np.float64))
    assert direct.rel_l2(m.grad.double().cpu().numpy(), ref) < 1e-5
    op.close()


# the multi-right-hand-side workload: N_t = 256, N_d = 200, N_m = 50 000, 64 vectors
PICK = [0, 21, 42, 63]


@pytest.fixture(scope="module")
def multi_rhs():
    from tests.test_gpu_fullsize import device_blocks, device_normals
    w = synth.WORKLOADS["multi-rhs"]
    blocks = device_blocks(w)
    m = device_normals(w, synth.workloads.T_PARAM, (w.nrhs, w.N_t, w.N_m))
    wt = device_normals(w, synth.workloads.T_WEIGHTS, (w.nrhs, w.N_t, w.N_d))
    src = lambda k: blocks[k].cpu().numpy()
    ref = direct.adjoint(src, wt[PICK].double().cpu().numpy(), w.N_t)   # the oracle's transpose
    yield w, blocks, m, wt, ref
    del blocks
    torch.cuda.empty_cache()


# (format, products, tolerance of the gradient against the oracle, finite-difference step, its tolerance).
# A linear loss makes the central difference exact for any step up to rounding; the perturbation
# h v must stay above the rounding of the perturbed spectra, or the difference measures that
# rounding instead of the derivative: BF16 spectra round at 2^-8 relative, above h = 1e-3, so the
# BF16 path takes h = 1; the split pair rounds at ~2^-17 (expected difference error ~3e-3 at
# h = 1e-3, ~3e-6 at h = 1); FP32 at 2^-24.  In units of ||grad||: L(m +- h v) carries a
# rounding error of about eps ||F m|| (eps the products' relative l2 error, ~8e-7 in FP32 at
# this workload), and ||F m|| ~ ||F* w|| for these iid vectors, so the FP32 difference at
# h = 1e-3 scatters by about 0.7 eps / h = 5.4e-4 per direction (measured 3e-5 .. 1.0e-3 over
# the 8 directions); 3e-3 is about 5.5 standard deviations.
MULTI = [("bf16", "tensor", 1e-2, 1.0, 1e-2), ("bf16x2", "tensor", 1e-5, 1e-3, 1e-2),
         ("bf16x2", "tensor", 1e-5, 1.0, 1e-4), ("f32", "simt", 1e-5, 1e-3, 3e-3)]


@pytest.mark.parametrize("prec,gemm,tol,h,fd_tol", MULTI, ids=["bf16-h1", "bf16x2-h1e-3", "bf16x2-h1", "f32-h1e-3"])
def test_multi_rhs_backward(multi_rhs, prec, gemm, tol, h, fd_tol):
    """The 64-vector workload through apply_F on the tensor cores (BF16, and
    the BF16 hi+lo split pair) and on the FP32 SIMT kernels: the gradient of
    L(m) = <w, F m> is the hand-written F* of w, checked on whole vectors 0,
    21, 42, 63 against the oracle's transpose, and by central differences of
    L (accumulated in FP64) along 8 random 64-vector directions."""
    w, blocks, m, wt, ref = multi_rhs
    op = btt.Operator(blocks, precision=prec, max_nrhs=w.nrhs, gemm=gemm)
    x = m.clone().requires_grad_(True)
    loss = (apply_F(op, x).double() * wt.double()).sum()
    loss.backward()
    op.device_status()
    grad = x.grad
    for n, b in enumerate(PICK):
        assert direct.rel_l2(grad[b].double().cpu().numpy(), ref[n]) < tol, b

    def L(v):
        return float((op.matvec(v).double() * wt.double()).sum())

    # <grad, v> for v with iid N(0,1) entries has standard deviation ||grad||:
    # the differences are compared on that scale
    scale = float(torch.linalg.vector_norm(grad.double()))
    gen = synth.dev_lib()
    for k in range(8):
        v = torch.empty_like(m)
        assert gen.synth_dev_normal(w.seed + 100 + k, synth.workloads.T_DIRS, 0, v.numel(), None, v.data_ptr(),
                                    None) == 0
        fd = (L(m + h * v) - L(m - h * v)) / (2 * h)
        an = float((grad.double() * v.double()).sum())
        assert abs(fd - an) <= fd_tol * scale, (k, fd, an, scale)
        del v
    op.close()
    del x, grad
    torch.cuda.empty_cache()
