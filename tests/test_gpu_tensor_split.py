"""BF16 hi+lo split pairs on the tensor cores: each product is
A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation, where B is the
stored Fhat pair and A the BF16 pair of the FP32 spectra.

Two bars, as for single BF16: (1) against the exact operator, the split
pair's tolerance 1e-5; (2) against the oracle's algorithm applied to the
same rounded operands with the same three products (oracle/quantize.py
rounding, the lo*lo term left out), where only FP32 accumulation over
2 ldm x 3 terms remains (measured 2.3e-6 at K = 672; bound 8e-6, while a
lo plane that is wrong or missing leaves BF16-level error, ~1e-3).  (2) pins the second operand planes: a lo tile from the wrong
plane or offset, or a missing cross product, would miss it by orders of
magnitude while possibly still passing (1) loosely."""
import numpy as np
import pytest
import torch

import synth
from oracle import direct, fft_method, quantize
import paper_2407_13066_gb300 as btt

pytestmark = pytest.mark.gpu


def split(z):
    """BF16 hi and lo pairs of complex values rounded to FP32 first."""
    z = z.astype(np.complex64).astype(np.complex128)
    hi = quantize.to_bf16(z.real) + 1j * quantize.to_bf16(z.imag)
    r = (z - hi).astype(np.complex64).astype(np.complex128)
    lo = quantize.to_bf16(r.real) + 1j * quantize.to_bf16(r.imag)
    return hi, lo


def fhat_pair(F):
    Fh = fft_method.setup(F)
    hi = quantize.to_bf16(Fh.real) + 1j * quantize.to_bf16(Fh.imag)
    r = (Fh - hi).astype(np.complex64).astype(np.complex128)
    lo = quantize.to_bf16(r.real) + 1j * quantize.to_bf16(r.imag)
    return hi, lo


def three_products(apply, Fhi, Flo, xhi, xlo):
    return apply(Fhi, xhi) + apply(Flo, xhi) + apply(Fhi, xlo)


def rounded_forward(F, m):
    Fhi, Flo = fhat_pair(F)
    xhi, xlo = split(fft_method.transform(m))
    return fft_method.inverse_transform(three_products(fft_method.apply_fhat, Fhi, Flo, xhi, xlo), m.shape[-2])


def rounded_adjoint(F, d):
    Fhi, Flo = fhat_pair(F)
    yhi, ylo = split(fft_method.transform(d))
    return fft_method.inverse_transform(three_products(fft_method.apply_fhat_adjoint, Fhi, Flo, yhi, ylo),
                                        d.shape[-2])


def run(w, nrhs, action, gemm="tensor", max_nrhs=None):
    F = synth.blocks(w)
    m = synth.vectors(w, "m", nrhs).astype(np.float32).astype(np.float64)
    d = synth.vectors(w, "d", nrhs).astype(np.float32).astype(np.float64)
    g = synth.noise_gamma_inv(w).astype(np.float32).astype(np.float64)
    with btt.Operator(F, precision="bf16x2", max_nrhs=max_nrhs or nrhs, gemm=gemm) as op:
        if action == "matvec":
            out = op.matvec(torch.from_numpy(m.astype(np.float32)).cuda())
        elif action == "adjoint":
            out = op.adjoint(torch.from_numpy(d.astype(np.float32)).cuda())
        else:
            out = op.hessian(torch.from_numpy(m.astype(np.float32)).cuda(),
                             torch.from_numpy(g.astype(np.float32)).cuda())
        op.device_status()
        got = out.double().cpu().numpy()
    return F, m, d, g, got


SHAPES = [
    ((64, 8, 32), 16),          # one K tile, tiny N
    ((96, 50, 333), 64),        # ragged K, N_d = 50 -> N = 64
    ((128, 200, 700), 70),      # two 64-vector launches (64 + 6), N = 208
    ((60, 300, 150), 20),       # two N tiles of 160 rows
    ((128, 16, 6000), 16),      # 188 K tiles in 7 splits of 27: two accumulation chains per CTA (24 + 3)
]


@pytest.mark.parametrize("shape,nrhs", SHAPES)
def test_split_tensor_matvec(shape, nrhs):
    N_t, N_d, N_m = shape
    w = synth.Workload("tcs", N_t, N_d, N_m, tau=N_t / 5, seed=N_d + N_m)
    F, m, _, _, got = run(w, nrhs, "matvec")
    assert direct.rel_l2(got, direct.forward(F, m)) < 1e-5
    assert direct.rel_l2(got, rounded_forward(F, m)) < 8e-6


@pytest.mark.parametrize("shape,nrhs", SHAPES)
def test_split_tensor_adjoint(shape, nrhs):
    N_t, N_d, N_m = shape
    w = synth.Workload("tcsa", N_t, N_d, N_m, tau=N_t / 5, seed=N_d + 3 * N_m)
    F, _, d, _, got = run(w, nrhs, "adjoint")
    assert direct.rel_l2(got, direct.adjoint(F, d)) < 1e-5
    assert direct.rel_l2(got, rounded_adjoint(F, d)) < 8e-6


def test_split_tensor_hessian_and_chunking():
    w = synth.Workload("tcsh", 100, 60, 400, tau=20.0, seed=12)
    F, m, _, g, got = run(w, 40, "hessian", max_nrhs=24)
    assert direct.rel_l2(got, direct.hessian(F, m, g)) < 1e-5


def test_split_tensor_matches_simt():
    w = synth.Workload("tcs2", 80, 40, 500, tau=16.0, seed=2)
    F, m, _, _, tc = run(w, 32, "matvec")
    _, _, _, _, simt = run(w, 32, "matvec", gemm="simt")
    exact = direct.forward(F, m)
    assert direct.rel_l2(simt, exact) < 1e-5 and direct.rel_l2(tc, exact) < 1e-5
    assert direct.rel_l2(tc, simt) < 1e-5
