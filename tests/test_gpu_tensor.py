"""Multi-right-hand-side products on the tensor cores (tcgen05, BF16 in,
FP32 accumulate) against the FP64 oracle.

Two bars: (1) against the exact operator, the BF16 tolerance 1e-2;
(2) against the oracle's own algorithm applied to the same rounded inputs
-- Fhat rounded to BF16 (oracle/quantize.py), the spectra of m (or d)
rounded to FP32 then BF16, as the tensor-core operand is, and the
adjoint's output spectra rounded to BF16, as the adjoint hands them to the
inverse transform -- where only FP32 accumulation error remains, plus the
rare output spectrum that FP32 accumulation and the FP64 reference round
to neighbouring BF16 values (1e-4).  (2) pins the operand layouts and the
complex-to-real mapping; a transposed tile or a dropped imaginary term
would miss it by orders of magnitude.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import direct, fft_method, quantize
import paper_2407_13066_gb300 as btt

pytestmark = pytest.mark.gpu


def rounded_reference(F, m):
    """Alg. 2 in FP64 on BF16 Fhat and BF16 spectra (FP32 first)."""
    Fh = quantize.quantize(fft_method.setup(F), "bf16")
    mh = fft_method.transform(m)
    mh = quantize.to_bf16(mh.real) + 1j * quantize.to_bf16(mh.imag)
    return fft_method.inverse_transform(fft_method.apply_fhat(Fh, mh), m.shape[-2])


def bf16c(z):
    z = z.astype(np.complex64)
    return quantize.to_bf16(z.real) + 1j * quantize.to_bf16(z.imag)


def rounded_adjoint(F, d):
    """Alg. 3 in FP64 on BF16 Fhat and BF16 (FP32 first) data spectra; the
    output spectra rounded to BF16 before the inverse transform."""
    Fh = quantize.quantize(fft_method.setup(F), "bf16")
    mh = bf16c(fft_method.apply_fhat_adjoint(Fh, bf16c(fft_method.transform(d))))
    return fft_method.inverse_transform(mh, d.shape[-2])


def rounded_hessian(F, m, g):
    Fh = quantize.quantize(fft_method.setup(F), "bf16")
    N_t = m.shape[-2]
    d = fft_method.inverse_transform(fft_method.apply_fhat(Fh, bf16c(fft_method.transform(m))), N_t) * g
    mh = bf16c(fft_method.apply_fhat_adjoint(Fh, bf16c(fft_method.transform(d))))
    return fft_method.inverse_transform(mh, N_t)


def run(w, nrhs, gemm, max_nrhs=None, action="matvec"):
    F = synth.blocks(w)
    m = synth.vectors(w, "m", nrhs).astype(np.float32).astype(np.float64)
    d = synth.vectors(w, "d", nrhs).astype(np.float32).astype(np.float64)
    g = synth.noise_gamma_inv(w).astype(np.float32).astype(np.float64)
    with btt.Operator(F, precision="bf16", max_nrhs=max_nrhs or nrhs, gemm=gemm) as op:
        mt = torch.from_numpy(m.astype(np.float32)).cuda()
        if action == "matvec":
            out = op.matvec(mt)
        elif action == "adjoint":
            out = op.adjoint(torch.from_numpy(d.astype(np.float32)).cuda())
        else:
            out = op.hessian(mt, torch.from_numpy(g.astype(np.float32)).cuda())
        op.device_status()
        got = out.double().cpu().numpy()
    if action == "adjoint":
        return F, d, g, got
    return F, m, g, got


@pytest.mark.parametrize("shape,nrhs", [
    ((64, 8, 32), 16),          # one K tile, tiny N
    ((96, 50, 333), 64),        # ragged K (2*336 = 672 = 10.5 tiles), N_d = 50 -> N = 64
    ((128, 200, 700), 70),      # two M tiles (64 + 6), N = 208
    ((60, 300, 150), 20),       # two N tiles of 160 rows
    ((100, 24, 2000), 130),     # three launches of <= 128 vectors, many K splits
])
def test_tensor_matvec(shape, nrhs):
    N_t, N_d, N_m = shape
    w = synth.Workload("tc", N_t, N_d, N_m, tau=N_t / 5, seed=N_d + N_m)
    F, m, _, got = run(w, nrhs, "tensor")
    assert direct.rel_l2(got, direct.forward(F, m)) < 1e-2
    assert direct.rel_l2(got, rounded_reference(F, m)) < 1e-4


@pytest.mark.parametrize("shape,nrhs", [
    ((64, 8, 32), 16),          # one K tile (N_d = 8), one column tile
    ((96, 50, 333), 64),        # ragged columns (2*336 = 672 reals = 2.6 tiles)
    ((128, 200, 700), 70),      # K = 200 over 4 tiles, two launches of 64 vectors
    ((60, 300, 150), 20),       # K = 300 over 5 tiles
])
def test_tensor_adjoint(shape, nrhs):
    N_t, N_d, N_m = shape
    w = synth.Workload("tca", N_t, N_d, N_m, tau=N_t / 5, seed=N_d + 3 * N_m)
    F, d, _, got = run(w, nrhs, "tensor", action="adjoint")
    assert direct.rel_l2(got, direct.adjoint(F, d)) < 1e-2
    assert direct.rel_l2(got, rounded_adjoint(F, d)) < 1e-4


def test_tensor_hessian_both_passes():
    w = synth.Workload("tch", 100, 60, 400, tau=20.0, seed=12)
    F, m, g, got = run(w, 33, "tensor", action="hessian")
    assert direct.rel_l2(got, direct.hessian(F, m, g)) < 1e-2
    # Two BF16 roundings here follow FP32 arithmetic on the device and FP64
    # in the reference (the data spectra after the forward pass and the
    # middle step, the output spectra of the adjoint); where the two land on
    # neighbouring BF16 values the entry moves by one BF16 step (2^-8
    # relative).  A fraction p of such entries gives ~sqrt(p) 2^-8: measured
    # 2.8e-4.  A layout or mapping mistake gives O(1).
    assert direct.rel_l2(got, rounded_hessian(F, m, g)) < 1e-3


def test_tensor_matches_simt_within_bf16_spectra_rounding():
    w = synth.Workload("tc2", 80, 40, 500, tau=16.0, seed=2)
    _, m, _, tc = run(w, 32, "tensor")
    F, _, _, simt = run(w, 32, "simt")
    assert direct.rel_l2(tc, simt) < 5e-3
    exact = direct.forward(F, m)
    assert direct.rel_l2(simt, exact) < 1e-2 and direct.rel_l2(tc, exact) < 1e-2


def test_tensor_hessian_and_chunking():
    w = synth.Workload("tc3", 50, 30, 256, tau=10.0, seed=4)
    F, m, g, got = run(w, 40, "tensor", max_nrhs=24, action="hessian")
    assert direct.rel_l2(got, direct.hessian(F, m, g)) < 1e-2


def test_auto_mode_picks_by_batch():
    w = synth.Workload("tc4", 32, 16, 64, tau=8.0, seed=6)
    F, m, _, a = run(w, 20, "auto")      # >= 16 right-hand sides: tensor cores
    _, _, _, b = run(w, 20, "tensor")
    np.testing.assert_array_equal(a, b)
    _, _, _, c = run(w, 4, "auto")       # few: SIMT kernels
    _, _, _, d = run(w, 4, "simt")
    np.testing.assert_array_equal(c, d)
