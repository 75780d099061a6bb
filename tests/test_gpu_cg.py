"""Conjugate gradients on the device (btt_cg) against a dense FP64 solve of
the regularised normal equations (H + alpha I) x = b, H = F^T Gamma^-1 F
(Sec. 2.2, Eq. LinearInverseProblem with R = I)."""
import numpy as np
import pytest
import torch

import synth
import paper_2407_13066_gb300 as btt
from tests.test_oracle_pins import dense_matrix

pytestmark = pytest.mark.gpu


def system(N_t, N_d, N_m, seed):
    w = synth.Workload("cg", N_t, N_d, N_m, tau=N_t / 4, seed=seed)
    F = synth.blocks(w)
    g = synth.noise_gamma_inv(w).astype(np.float32)
    A = dense_matrix(F)
    H = A.T @ (g.astype(np.float64).ravel()[:, None] * A)
    lam = np.linalg.eigvalsh(H).max()
    return w, F, g, H, lam


# 2 N_t = 80 has no fixed transform plan (the CG step runs as its own
# kernel); 2 N_t = 128 has one (the step runs inside the Hessian's last
# inverse transform)
@pytest.mark.parametrize("N_t", [40, 64])
@pytest.mark.parametrize("prec,gemm,tol,bound", [("f32", "simt", 1e-6, 2e-4), ("bf16", "tensor", 1e-3, 2e-2)])
def test_cg_matches_dense_solve(prec, gemm, tol, bound, N_t):
    w, F, g, H, lam = system(N_t, 6, 30, 5)
    alpha = lam / 50.0                       # condition number <= 51
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


def test_cg_warm_start_and_zero_rhs():
    w, F, g, H, lam = system(16, 4, 12, 9)
    alpha = lam / 10.0
    b = synth.vectors(w, "m", 1).astype(np.float32)
    ref = np.linalg.solve(H + alpha * np.eye(H.shape[0]), b[0].astype(np.float64).ravel()).reshape(b.shape[1:])
    with btt.Operator(F, precision="f32") as op:
        x0 = torch.from_numpy(ref.astype(np.float32)[None]).cuda()
        x, its, rel = op.cg(torch.from_numpy(b).cuda(), alpha, gamma_inv=torch.from_numpy(g).cuda(), x0=x0,
                            tol=1e-4, max_iter=100)
        assert its[0] <= 2                     # started at the solution
        z, its0, rel0 = op.cg(torch.zeros_like(x), alpha, tol=1e-6)
        assert its0 == [0] and float(z.abs().max()) == 0.0


def test_cg_matches_oracle_cg():
    """Against the FP64 CPU CG of the oracle on an operator too large to
    assemble (n = N_t N_m = 64 000 unknowns, several FFT tiles and a ragged
    tail): same solution to the solver tolerance, similar iteration count."""
    from oracle import cg as ocg
    from oracle import fft_method
    w = synth.Workload("cg-large", 128, 10, 500, tau=32.0, seed=6)
    F = synth.blocks(w)
    g = synth.noise_gamma_inv(w)
    Fhat = fft_method.setup(F)
    v = synth.vectors(w, "m", 1, tensor_id=synth.workloads.T_DIRS)[0]
    for _ in range(30):                      # power iteration for the top eigenvalue
        v = fft_method.hessian(Fhat, v, g)
        lam = np.linalg.norm(v)
        v /= lam
    alpha = lam / 40.0
    b = synth.vectors(w, "m", 2).astype(np.float32)
    tol = 1e-5
    refs = [ocg.solve_regularised(Fhat, b[j].astype(np.float64), alpha, g, tol=tol, max_iter=300) for j in range(2)]
    with btt.Operator(F, precision="f32", max_nrhs=2) as op:
        x, its, rel = op.cg(torch.from_numpy(b).cuda(), alpha, gamma_inv=torch.from_numpy(g.astype(np.float32)).cuda(),
                            tol=tol, max_iter=300)
        op.device_status()
    x = x.double().cpu().numpy()
    for j, (xr, itr, relr) in enumerate(refs):
        assert relr <= tol and rel[j] <= tol
        assert abs(its[j] - itr) <= max(3, itr // 5), (its[j], itr)
        err = np.linalg.norm(x[j] - xr) / np.linalg.norm(xr)
        assert err < 40 * tol, err


def test_cg_fused_step_in_chunks():
    """More right-hand sides than the operator's batch workspace (max_nrhs
    2, 5 vectors): the Hessian runs in chunks of 2, 2, 1 and the CG step
    fused into its last inverse transform (2 N_t = 128 has a fixed plan)
    must address each chunk's x, r, p, scalars and partial sums.  Every
    vector matches the dense solve, and equals its solve alone."""
    w, F, g, H, lam = system(64, 6, 30, 7)
    alpha = lam / 50.0
    nrhs = 5
    b = synth.vectors(w, "m", nrhs).astype(np.float32)
    ref = np.stack([np.linalg.solve(H + alpha * np.eye(H.shape[0]), b[j].astype(np.float64).ravel())
                    for j in range(nrhs)]).reshape(b.shape)
    gt = torch.from_numpy(g).cuda()
    with btt.Operator(F, precision="f32", max_nrhs=2) as op:
        x, its, rel = op.cg(torch.from_numpy(b).cuda(), alpha, gamma_inv=gt, tol=1e-6, max_iter=400)
        x3, its3, _ = op.cg(torch.from_numpy(b[3:4]).cuda(), alpha, gamma_inv=gt, tol=1e-6, max_iter=400)
        op.device_status()
    x = x.double().cpu().numpy()
    assert all(r <= 1e-6 for r in rel), rel
    for j in range(nrhs):
        err = np.linalg.norm(x[j] - ref[j]) / np.linalg.norm(ref[j])
        assert err < 2e-4, (j, err)
    # a vector's run does not depend on the others in its batch
    assert its3[0] == its[3]
    assert np.array_equal(x3.double().cpu().numpy()[0], x[3])
