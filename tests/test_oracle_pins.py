"""Pins of the FP64 oracle to facts outside itself.

Each test fixes the oracle against something the paper or mathematics
determines: a hand-worked example, the dense matrix of Eq. ShiftInvariance
assembled block by block, the textbook scalar convolution (Sec. 2.4), the
adjoint identity, shift invariance, closed forms for identity, single-lag
and geometric rank-1 operators, and a second independent implementation
(naive C loops).  test_oracle_mutants.py shows that plausible mistakes
planted in the oracle fail these pins.
"""
import os

import numpy as np
import pytest

import synth
from oracle import direct, fft_method, naive, quantize

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def _golden():
    cases = {}
    with open(os.path.join(GOLDEN, "toeplitz_hand.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                c, key, *vals = line.split()
                cases.setdefault(c, {})[key] = np.array([float(v) for v in vals])
    return cases


def dense_matrix(F):
    """Eq. ShiftInvariance written out: block (i, j) is F_{i-j} for i >= j."""
    N_t, N_d, N_m = F.shape
    A = np.zeros((N_t * N_d, N_t * N_m))
    for i in range(N_t):
        for j in range(i + 1):
            A[i * N_d:(i + 1) * N_d, j * N_m:(j + 1) * N_m] = F[i - j]
    return A


def rand_op(N_t, N_d, N_m, nrhs=None):
    F = RNG.standard_normal((N_t, N_d, N_m))
    shp = () if nrhs is None else (nrhs,)
    return F, RNG.standard_normal(shp + (N_t, N_m)), RNG.standard_normal(shp + (N_t, N_d))


ALL_FORWARD = {
    "direct": lambda F, m: direct.forward(F, m),
    "naive": lambda F, m: naive.forward(F, m),
    "fft": lambda F, m: fft_method.forward(fft_method.setup(F), m),
}
ALL_ADJOINT = {
    "direct": lambda F, d: direct.adjoint(F, d),
    "naive": lambda F, d: naive.adjoint(F, d),
    "fft": lambda F, d: fft_method.adjoint(fft_method.setup(F), d),
}


@pytest.mark.parametrize("impl", list(ALL_FORWARD))
def test_hand_worked_examples(impl):
    g = _golden()
    A, B = g["A"], g["B"]
    F = A["f"].reshape(4, 1, 1)
    np.testing.assert_allclose(ALL_FORWARD[impl](F, A["x"].reshape(4, 1)).ravel(), A["Fx"], atol=1e-12)
    np.testing.assert_allclose(ALL_ADJOINT[impl](F, A["y"].reshape(4, 1)).ravel(), A["FTy"], atol=1e-12)
    F = np.stack([B["F0"].reshape(1, 2), B["F1"].reshape(1, 2)])
    np.testing.assert_allclose(ALL_FORWARD[impl](F, B["m"].reshape(2, 2)).ravel(), B["Fm"], atol=1e-12)
    np.testing.assert_allclose(ALL_ADJOINT[impl](F, B["d"].reshape(2, 1)).ravel(), B["FTd"], atol=1e-12)


@pytest.mark.parametrize("impl", list(ALL_FORWARD))
@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 3, 4), (7, 2, 9), (6, 5, 1), (1, 4, 3)])
def test_dense_matrix(impl, shape):
    F, m, d = rand_op(*shape)
    A = dense_matrix(F)
    np.testing.assert_allclose(ALL_FORWARD[impl](F, m).ravel(), A @ m.ravel(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ALL_ADJOINT[impl](F, d).ravel(), A.T @ d.ravel(), rtol=1e-12, atol=1e-12)


def test_dense_matrix_fp64_small_workload():
    w = synth.WORKLOADS["fp64-small"]
    F = synth.blocks(w)
    m = synth.vectors(w, "m")[0]
    d = synth.vectors(w, "d")[0]
    A = dense_matrix(F)
    ref_d, ref_m = A @ m.ravel(), A.T @ d.ravel()
    assert direct.rel_l2(direct.forward(F, m).ravel(), ref_d) < 1e-14
    assert direct.rel_l2(direct.adjoint(F, d).ravel(), ref_m) < 1e-14
    assert direct.rel_l2(naive.forward(F, m).ravel(), ref_d) < 1e-14
    assert direct.rel_l2(fft_method.forward(fft_method.setup(F), m).ravel(), ref_d) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_scalar_case_is_truncated_convolution(n):
    """N_d = N_m = 1: a lower-triangular Toeplitz matrix (Sec. 2.4) is the
    first n terms of the linear convolution of its first column with x."""
    f, x = RNG.standard_normal(n), RNG.standard_normal(n)
    ref = np.convolve(f, x)[:n]
    for impl in ALL_FORWARD.values():
        np.testing.assert_allclose(impl(f.reshape(n, 1, 1), x.reshape(n, 1)).ravel(), ref,
                                   rtol=1e-12, atol=1e-12)
    # the transpose is the correlation: (F^T y)_j = sum_{i>=j} f_{i-j} y_i
    y = RNG.standard_normal(n)
    ref_t = np.correlate(y, f, mode="full")[n - 1:]
    for impl in ALL_ADJOINT.values():
        np.testing.assert_allclose(impl(f.reshape(n, 1, 1), y.reshape(n, 1)).ravel(), ref_t,
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 3, 5), (33, 4, 2), (64, 8, 32)])
def test_adjoint_identity(shape):
    F, m, d = rand_op(*shape)
    for name in ALL_FORWARD:
        lhs = np.vdot(ALL_FORWARD[name](F, m), d)
        rhs = np.vdot(m, ALL_ADJOINT[name](F, d))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)) * np.sqrt(m.size)


@pytest.mark.parametrize("shift", [1, 3, 9])
def test_shift_invariance(shift):
    F, m, d = rand_op(12, 3, 4)
    ms = np.zeros_like(m)
    ms[shift:] = m[:-shift]
    for impl in ALL_FORWARD.values():
        ds, d0 = impl(F, ms), impl(F, m)
        np.testing.assert_allclose(ds[shift:], d0[:-shift], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(ds[:shift], 0.0, atol=1e-12)
    # the adjoint is shift-invariant the other way
    dsh = np.zeros_like(d)
    dsh[:-shift] = d[shift:]
    for impl in ALL_ADJOINT.values():
        a, b = impl(F, dsh), impl(F, d)
        np.testing.assert_allclose(a[:-shift], b[shift:], rtol=1e-12, atol=1e-12)


def test_identity_block():
    N = 6
    F = np.zeros((10, N, N))
    F[0] = np.eye(N)
    _, m, d = rand_op(10, N, N)
    for name in ALL_FORWARD:
        np.testing.assert_allclose(ALL_FORWARD[name](F, m), m, atol=1e-13)
        np.testing.assert_allclose(ALL_ADJOINT[name](F, d), d, atol=1e-13)


@pytest.mark.parametrize("lag", [0, 1, 5, 9])
def test_single_nonzero_block(lag):
    N_t, N_d, N_m = 10, 3, 4
    G = RNG.standard_normal((N_d, N_m))
    F = np.zeros((N_t, N_d, N_m))
    F[lag] = G
    _, m, d = rand_op(N_t, N_d, N_m)
    ref_d = np.zeros((N_t, N_d))
    ref_d[lag:] = m[: N_t - lag] @ G.T          # d_i = G m_{i-lag}
    ref_m = np.zeros((N_t, N_m))
    ref_m[: N_t - lag] = d[lag:] @ G            # m_j = G^T d_{j+lag}
    for name in ALL_FORWARD:
        np.testing.assert_allclose(ALL_FORWARD[name](F, m), ref_d, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(ALL_ADJOINT[name](F, d), ref_m, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("r", [0.5, 0.97, -0.8])
def test_geometric_rank_one_closed_form(r):
    """F_k = r^k u v^T and m_j = v for all j give
    d_i = |v|^2 u (1 - r^{i+1}) / (1 - r)."""
    N_t, N_d, N_m = 40, 5, 7
    u, v = RNG.standard_normal(N_d), RNG.standard_normal(N_m)
    F = np.stack([r ** k * np.outer(u, v) for k in range(N_t)])
    m = np.tile(v, (N_t, 1))
    i = np.arange(N_t)
    ref = (v @ v) * np.outer((1 - r ** (i + 1)) / (1 - r), u)
    for impl in ALL_FORWARD.values():
        np.testing.assert_allclose(impl(F, m), ref, rtol=1e-11, atol=1e-11)


def test_hessian_properties():
    F, m, _ = rand_op(16, 4, 6)
    m2 = RNG.standard_normal(m.shape)
    g = RNG.uniform(0.5, 2.0, (16, 4))
    H = lambda x: direct.hessian(F, x, g)
    assert abs(np.vdot(H(m), m2) - np.vdot(m, H(m2))) < 1e-10 * np.linalg.norm(m) * np.linalg.norm(m2)
    assert np.vdot(H(m), m) > 0
    np.testing.assert_allclose(direct.hessian(F, m), direct.adjoint(F, direct.forward(F, m)), rtol=1e-13)
    # dense: H = A^T diag(g) A
    A = dense_matrix(F)
    np.testing.assert_allclose(H(m).ravel(), A.T @ (g.ravel() * (A @ m.ravel())), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(fft_method.hessian(fft_method.setup(F), m, g), H(m), rtol=1e-11, atol=1e-11)


def test_batched_rhs_equal_single():
    F, m, d = rand_op(9, 3, 5, nrhs=4)
    for b in range(4):
        np.testing.assert_allclose(direct.forward(F, m)[b], naive.forward(F, m[b]), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(direct.adjoint(F, d)[b], naive.adjoint(F, d[b]), rtol=1e-12, atol=1e-12)


def test_block_callable_and_sampled_entries():
    w = synth.Workload("t", 20, 5, 11, tau=7.0, envelope=True, seed=4)
    F = synth.blocks(w)
    m = synth.vectors(w, "m")[0]
    d = synth.vectors(w, "d")[0]
    full_d = direct.forward(F, m)
    np.testing.assert_allclose(direct.forward(lambda k: synth.blocks(w, k, k + 1)[0], m), full_d, rtol=1e-14)
    samples = [(0, 0), (19, 4), (7, 2), (13, 0)]
    row_fn = lambda ks, s: synth.block_entries(w, ks[:, None], s, np.arange(w.N_m)[None, :])
    got = direct.forward_entries(row_fn, m, samples)
    np.testing.assert_allclose(got, [full_d[i, s] for i, s in samples], rtol=1e-13)
    full_m = direct.adjoint(F, d)
    col_fn = lambda ks, l: synth.block_entries(w, ks[:, None], np.arange(w.N_d)[None, :], l)
    samples = [(0, 0), (19, 10), (5, 3)]
    got = direct.adjoint_entries(col_fn, d, samples)
    np.testing.assert_allclose(got, [full_m[j, l] for j, l in samples], rtol=1e-13)


def test_fft_readings():
    """Sec. 2.4 embedding: F-hat has N_t + 1 slices; w = 0 and w = N_t are
    real; the forward DFT is unnormalised (slice 0 is the sum over lags)."""
    F, _, _ = rand_op(10, 2, 3)
    Fh = fft_method.setup(F)
    assert Fh.shape == (11, 2, 3)
    np.testing.assert_allclose(Fh[0].real, F.sum(0), rtol=1e-13)
    np.testing.assert_allclose(Fh[0].imag, 0, atol=1e-13)
    np.testing.assert_allclose(Fh[10].imag, 0, atol=1e-12)
    np.testing.assert_allclose(Fh[10].real, (F * (-1.0) ** np.arange(10)[:, None, None]).sum(0), rtol=1e-12)


def test_quantize_formats():
    F, _, _ = rand_op(32, 4, 6)
    Fh = fft_method.setup(F)
    scale = np.abs(Fh).max()
    for fmt, tol in [("fp32", 1e-7), ("fp16s", 1e-3), ("bf16", 8e-3), ("bf16x2", 2e-5)]:
        q = quantize.quantize(Fh, fmt)
        err = np.abs(q - Fh).max() / scale
        assert err < tol, (fmt, err)
    # bf16 rounding is to nearest even: 1 + 2^-8 (a tie) rounds down to 1,
    # 1 + 3*2^-8 (a tie) rounds up to 1 + 2^-6... of spacing 2^-7
    assert quantize.to_bf16(1.0 + 2.0 ** -8) == 1.0
    assert quantize.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # E4M3: nearest even at ties, subnormal spacing 2^-9, saturation at 448
    e = quantize.to_e4m3
    assert e(1.0) == 1.0 and e(1.0625) == 1.0 and e(1.1875) == 1.25
    assert e(0.3) == 0.3125 and e(-0.3) == -0.3125
    assert e(448.0) == 448.0 and e(460.0) == 448.0 and e(500.0) == 448.0 and e(1e9) == 448.0
    assert e(2.0 ** -9) == 2.0 ** -9 and e(2.0 ** -10) == 0.0 and e(3 * 2.0 ** -10) == 2.0 ** -8
    assert e(240.0) == 240.0 and e(247.9) == 240.0 and e(248.0) == 256.0
    codes = np.array([m * 2.0 ** k for k in range(-6, 9) for m in (1, 1.125, 1.25, 1.375, 1.5, 1.625, 1.75, 1.875)])
    codes = codes[codes <= 448]
    np.testing.assert_array_equal(e(codes), codes)     # every normal code is a fixed point
    q8 = quantize.quantize(Fh, "fp8s")
    assert np.abs(q8 - Fh).max() / scale < 0.07
    s8 = quantize.fp8_scales(Fh)
    assert np.all(np.abs(Fh.real) / s8[:, None, None] <= 256 * (1 + 1e-6))
    s = quantize.fp16_scales(Fh)
    assert s.shape == (33,)
    assert np.all(np.abs(Fh.real) / s[:, None, None] <= 16384 * (1 + 1e-6))
