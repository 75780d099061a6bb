"""Pins of the oracle's conjugate-gradient solve (oracle/cg.py) against
facts of the method itself: the exact solution of a dense system, finite
termination in as many steps as the operator has distinct eigenvalues, and
the regularised normal equations assembled densely.  Planted mistakes (no
conjugation, a wrong step length) must fail a pin."""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import fft_method
from tests.test_oracle_pins import dense_matrix

RNG = np.random.default_rng(11)


def _spd(n, cond):
    q, _ = np.linalg.qr(RNG.standard_normal((n, n)))
    return (q * np.geomspace(1.0, cond, n)) @ q.T


def test_dense_spd_solution():
    A = _spd(12, 50.0)
    b = RNG.standard_normal(12)
    x, it, rel = ocg.cg(lambda v: A @ v, b, tol=1e-13, max_iter=100)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    assert rel <= 1e-12 and it <= 12 + 3


def test_finite_termination_distinct_eigenvalues():
    """In exact arithmetic CG ends after as many iterations as A has distinct
    eigenvalues (with b touching all of them); 3 here, to rounding."""
    d = np.repeat([1.0, 4.0, 9.0], 20)
    q, _ = np.linalg.qr(RNG.standard_normal((60, 60)))
    A = (q * d) @ q.T
    b = RNG.standard_normal(60)
    x, it, rel = ocg.cg(lambda v: A @ v, b, tol=1e-10, max_iter=60)
    assert it == 3 and rel <= 1e-10


def test_zero_rhs_and_warm_start():
    A = _spd(8, 10.0)
    assert ocg.cg(lambda v: A @ v, np.zeros(8))[1] == 0
    b = RNG.standard_normal(8)
    x, it, _ = ocg.cg(lambda v: A @ v, b, tol=1e-10, x0=np.linalg.solve(A, b))
    assert it == 0


def test_regularised_normal_equations_match_dense():
    w = synth.Workload("cg-pin", 20, 4, 9, tau=5.0, seed=2)
    F = synth.blocks(w)
    g = synth.noise_gamma_inv(w)
    A = dense_matrix(F)
    alpha = 0.3
    H = A.T @ (g.ravel()[:, None] * A) + alpha * np.eye(A.shape[1])
    b = synth.vectors(w, "m", 1)[0]
    x, it, rel = ocg.solve_regularised(fft_method.setup(F), b, alpha, g, tol=1e-12, max_iter=500)
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(H, b.ravel()), rtol=1e-8, atol=1e-10)


def _steepest_descent(apply_A, b, tol=1e-8, max_iter=1000):
    x = np.zeros_like(b)
    r = b.copy()
    it = 0
    while it < max_iter and np.linalg.norm(r) > tol * np.linalg.norm(b):
        Ar = apply_A(r)
        x = x + (r @ r) / (r @ Ar) * r
        r = b - apply_A(x)
        it += 1
    return x, it, np.linalg.norm(r) / np.linalg.norm(b)


def _wrong_step(apply_A, b, tol=1e-8, max_iter=1000):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    it = 0
    while it < max_iter and np.sqrt(rr) > tol * np.linalg.norm(b):
        Ap = apply_A(p)
        a = rr / (p @ p)                      # should divide by p.Ap
        x, r = x + a * p, r - a * Ap
        rr, rr_old = r @ r, rr
        p = r + rr / rr_old * p
        it += 1
    return x, it, np.linalg.norm(b - apply_A(x)) / np.linalg.norm(b)


@pytest.mark.parametrize("mutant", [_steepest_descent, _wrong_step])
def test_mutants_fail_termination_pin(mutant):
    d = np.repeat([1.0, 4.0, 9.0], 20)
    q, _ = np.linalg.qr(RNG.standard_normal((60, 60)))
    A = (q * d) @ q.T
    b = RNG.standard_normal(60)
    _, it, rel = mutant(lambda v: A @ v, b, tol=1e-10, max_iter=60)
    assert not (it == 3 and rel <= 1e-10)
