"""torch.autograd through the operator: backward of F is the hand-written F*
kernel.  Checked by central finite differences (step 1e-3, 8 random
directions) of a linear loss L(m) = <w, F m>, accumulated in FP64 on the
host, and against the oracle's transpose."""
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
