"""Conjugate gradients in FP64 for (H + alpha I) x = b (TEST INFRASTRUCTURE).

Sec. 2.2 motivates the Hessian action F* Gamma^-1 F as the operator applied
inside an iterative (CG) solve of the regularised normal equations of
Eq. LinearInverseProblem; this is the textbook method of Hestenes and
Stiefel (1952), one right-hand side at a time, with the oracle's Hessian
(fft_method.hessian) as the operator.  Stops when ||r|| <= tol ||b|| or
after max_iter iterations.
"""
import numpy as np

from . import fft_method


def cg(apply_A, b, tol=1e-8, max_iter=1000, x0=None):
    """Solve A x = b for SPD A given as a function.  Returns (x, iterations,
    ||b - A x|| / ||b||) with the residual recomputed from x at the end."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - apply_A(x)
    p = r.copy()
    rr = float(np.vdot(r, r))
    it = 0
    while it < max_iter and np.sqrt(rr) > tol * bnorm:
        Ap = apply_A(p)
        a = rr / float(np.vdot(p, Ap))
        x = x + a * p
        r = r - a * Ap
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, float(np.linalg.norm(b - apply_A(x)) / bnorm)


def solve_regularised(Fhat, b, alpha, gamma_inv=None, tol=1e-8, max_iter=1000):
    """(F* Gamma^-1 F + alpha I) x = b for one parameter vector b [N_t][N_m]."""
    A = lambda v: fft_method.hessian(Fhat, v, gamma_inv) + alpha * v
    return cg(A, b, tol, max_iter)
