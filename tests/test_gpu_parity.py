"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances are relative l2 over the whole output against the FP64 oracle:
1e-12 for the FP64 operator, 1e-5 for FP32 storage and the BF16 hi+lo
pair, 2e-3 for FP16 with per-frequency scale, 1e-2 for BF16.  The reduced
formats are also checked far more tightly against the oracle's own
algorithm applied to the same rounded Fhat (oracle/quantize.py), which pins
the decode arithmetic rather than just the format's rounding.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import direct, fft_method, quantize
import paper_2407_13066_gb300 as btt

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16x2": 1e-5, "f16s": 2e-3, "bf16": 1e-2, "fp8s": 6e-2}
QFMT = {"f32": "fp32", "f16s": "fp16s", "bf16": "bf16", "bf16x2": "bf16x2", "fp8s": "fp8s"}


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def decode_e4m3(raw):
    """Value of each FP8 E4M3 byte (sign, 4 exponent bits bias 7, 3 mantissa)."""
    b = raw.astype(np.int64)
    sign = np.where(b & 0x80, -1.0, 1.0)
    ex = (b >> 3) & 0xF
    man = (b & 7).astype(np.float64)
    val = np.where(ex == 0, man / 8.0 * 2.0 ** -6, (1.0 + man / 8.0) * 2.0 ** (ex - 7))
    return sign * val


def inputs(w, nrhs=1, fp32=True):
    F = synth.blocks(w)
    m = synth.vectors(w, "m", nrhs)
    d = synth.vectors(w, "d", nrhs)
    g = synth.noise_gamma_inv(w)
    if fp32:  # the FP32 path sees FP32 inputs; the oracle uses the same values
        m, d, g = (a.astype(np.float32).astype(np.float64) for a in (m, d, g))
    return F, m, d, g


# ------------------------------------------------------------------ FP64
def test_fp64_small_workload_all_actions():
    w = synth.WORKLOADS["fp64-small"]
    F, m, d, g = inputs(w, fp32=False)
    with btt.Operator(torch.from_numpy(F).cuda(), precision="f64") as op:
        dm = host(op.matvec(dev(m[0], torch.float64)))
        md = host(op.adjoint(dev(d[0], torch.float64)))
        hm = host(op.hessian(dev(m[0], torch.float64), dev(g, torch.float64)))
    assert direct.rel_l2(dm, direct.forward(F, m[0])) < TOL["f64"]
    assert direct.rel_l2(md, direct.adjoint(F, d[0])) < TOL["f64"]
    assert direct.rel_l2(hm, direct.hessian(F, m[0], g)) < TOL["f64"]


def test_fp64_fhat_matches_oracle_setup():
    w = synth.WORKLOADS["fp64-small"]
    F = synth.blocks(w)
    with btt.Operator(F, precision="f64") as op:  # host blocks
        raw, _ = op.copy_fhat()
        ld = op.fhat_ld()
    got = raw.view(np.complex128).reshape(w.N_t + 1, w.N_d, ld)[:, :, :w.N_m]
    ref = fft_method.setup(F)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.all(raw.view(np.complex128).reshape(w.N_t + 1, w.N_d, ld)[:, :, w.N_m:] == 0)


# ---------------------------------------------------------- FP32 + shapes
SHAPES = [  # (N_t, N_d, N_m): single column, odd sizes, every radix, ragged tiles
    (1, 1, 1), (2, 3, 5), (3, 2, 7), (5, 4, 9), (7, 5, 3), (6, 9, 33), (30, 7, 517),
    (64, 8, 32), (105, 3, 70), (125, 13, 1001), (128, 1, 4), (252, 6, 260), (1000, 5, 130),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_shapes_all_actions(shape):
    N_t, N_d, N_m = shape
    w = synth.Workload("shape", N_t, N_d, N_m, tau=max(1.0, N_t / 4), seed=sum(shape))
    F, m, d, g = inputs(w, nrhs=2)
    with btt.Operator(torch.from_numpy(F).cuda(), precision="f32", max_nrhs=2) as op:
        dm = host(op.matvec(dev(m, torch.float32)))
        md = host(op.adjoint(dev(d, torch.float32)))
        hm = host(op.hessian(dev(m, torch.float32), dev(g, torch.float32)))
        h1 = host(op.hessian(dev(m, torch.float32)))
    assert direct.rel_l2(dm, direct.forward(F, m)) < TOL["f32"]
    assert direct.rel_l2(md, direct.adjoint(F, d)) < TOL["f32"]
    assert direct.rel_l2(hm, direct.hessian(F, m, g)) < TOL["f32"]
    assert direct.rel_l2(h1, direct.hessian(F, m)) < TOL["f32"]


def test_fp64_shapes():
    for N_t, N_d, N_m in [(1, 1, 1), (5, 4, 9), (105, 3, 70), (252, 6, 26)]:
        w = synth.Workload("s64", N_t, N_d, N_m, tau=N_t / 3 + 1, seed=N_t)
        F, m, d, g = inputs(w, nrhs=3, fp32=False)
        with btt.Operator(F, precision="f64", max_nrhs=2) as op:
            dm = host(op.matvec(dev(m, torch.float64)))
            md = host(op.adjoint(dev(d, torch.float64)))
            hm = host(op.hessian(dev(m, torch.float64), dev(g, torch.float64)))
        assert direct.rel_l2(dm, direct.forward(F, m)) < 1e-12
        assert direct.rel_l2(md, direct.adjoint(F, d)) < 1e-12
        assert direct.rel_l2(hm, direct.hessian(F, m, g)) < 1e-12


# --------------------------------------------------- reduced storage formats
@pytest.mark.parametrize("prec", ["f32", "f16s", "bf16", "bf16x2", "fp8s"])
def test_storage_formats(prec):
    w = synth.Workload("fmt", 96, 24, 300, tau=0.0, envelope=True, seed=5)
    F, m, d, g = inputs(w, nrhs=3)
    Fh = quantize.quantize(fft_method.setup(F), QFMT[prec])
    with btt.Operator(F, precision=prec, max_nrhs=4) as op:
        dm = host(op.matvec(dev(m, torch.float32)))
        md = host(op.adjoint(dev(d, torch.float32)))
        hm = host(op.hessian(dev(m, torch.float32), dev(g, torch.float32)))
    # against the exact operator, within the format's stated error
    assert direct.rel_l2(dm, direct.forward(F, m)) < TOL[prec]
    assert direct.rel_l2(md, direct.adjoint(F, d)) < TOL[prec]
    assert direct.rel_l2(hm, direct.hessian(F, m, g)) < TOL[prec]
    # against the same rounded Fhat: only FP32 arithmetic error remains
    assert direct.rel_l2(dm, fft_method.forward(Fh, m)) < 2e-6
    assert direct.rel_l2(md, fft_method.adjoint(Fh, d)) < 2e-6
    assert direct.rel_l2(hm, fft_method.hessian(Fh, m, g)) < 4e-6


@pytest.mark.parametrize("prec", ["f32", "f16s", "bf16", "bf16x2", "fp8s"])
def test_stored_fhat_matches_rounding_rule(prec):
    w = synth.Workload("fmt", 40, 6, 50, tau=10.0, envelope=True, seed=8)
    F = synth.blocks(w)
    ref = quantize.quantize(fft_method.setup(F), QFMT[prec])
    with btt.Operator(F, precision=prec) as op:
        raw, sc = op.copy_fhat()
        ld = op.fhat_ld()
    if prec == "f32":
        got = raw.view(np.complex64).astype(np.complex128)
    elif prec == "f16s":
        h = raw.view(np.float16).astype(np.float64).reshape(w.N_t + 1, -1) * sc[:, None].astype(np.float64)
        got = h[:, 0::2] + 1j * h[:, 1::2]
        np.testing.assert_allclose(sc, quantize.fp16_scales(fft_method.setup(F)), rtol=1e-6)
    elif prec == "fp8s":
        h = decode_e4m3(raw).reshape(w.N_t + 1, -1) * sc[:, None].astype(np.float64)
        got = h[:, 0::2] + 1j * h[:, 1::2]
        np.testing.assert_allclose(sc, quantize.fp8_scales(fft_method.setup(F)), rtol=1e-6)
    else:
        u = raw.view(np.uint16).astype(np.uint32) << 16
        f = u.view(np.float32).astype(np.float64)
        if prec == "bf16":
            got = f[0::2] + 1j * f[1::2]
        else:  # two planes: all hi pairs, then all lo pairs
            hi, lo = f[: f.size // 2], f[f.size // 2:]
            got = (hi[0::2] + lo[0::2]) + 1j * (hi[1::2] + lo[1::2])
    got = got.reshape(w.N_t + 1, w.N_d, ld)[:, :, :w.N_m]
    # one unit of the storage format at most (the FP64 transforms differ in rounding)
    ulp = {"f32": 2 ** -23, "f16s": 2 ** -10, "bf16": 2 ** -7, "bf16x2": 2 ** -15, "fp8s": 2 ** -3}[prec]
    assert np.abs(got - ref).max() <= ulp * np.abs(ref).max() * 1.01
    mism = np.mean(got != ref)
    assert mism < 0.01, mism


# ------------------------------------------------------- calling conventions
def test_host_and_device_pointers_agree():
    w = synth.Workload("ptr", 50, 7, 90, tau=12.0, seed=3)
    F, m, d, g = inputs(w, nrhs=5)
    with btt.Operator(torch.from_numpy(F), precision="f32", max_nrhs=2) as op:
        a = host(op.hessian(dev(m, torch.float32), dev(g, torch.float32)))
        b = op.hessian(m.astype(np.float32), g.astype(np.float32))          # pageable host
        pm = torch.from_numpy(m.astype(np.float32)).pin_memory()
        pg = torch.from_numpy(g.astype(np.float32)).pin_memory()
        out = torch.empty(pm.shape, dtype=torch.float32).pin_memory()
        op.hessian(pm, pg, out=out, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        c = out.double().numpy()
        e = host(op.matvec(dev(m, torch.float32)))
        f = op.matvec(m.astype(np.float32))
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(e, f)
    assert direct.rel_l2(a, direct.hessian(F, m, g)) < 1e-5


def test_batch_is_invariant():
    """A vector gives bit-identical results alone and in a batch (chunked or not)."""
    w = synth.Workload("batch", 64, 10, 200, tau=20.0, seed=9)
    F, m, d, _ = inputs(w, nrhs=7)
    res = {}
    for mx in (1, 3, 8):
        with btt.Operator(F, precision="f32", max_nrhs=mx) as op:
            res[mx] = (host(op.matvec(dev(m, torch.float32))), host(op.adjoint(dev(d, torch.float32))))
    single = res[1]
    for mx in (3, 8):
        # the per-frequency products accumulate each right-hand side in the
        # same order whatever the batch, but groups of 2/4 use other kernels
        for a, b in zip(res[mx], single):
            assert direct.rel_l2(a, b) < 1e-6
    assert direct.rel_l2(res[1][0], direct.forward(F, m)) < 1e-5


def test_zero_rhs_and_errors():
    w = synth.Workload("err", 8, 2, 3, tau=2.0)
    F = synth.blocks(w)
    op = btt.Operator(F, precision="f32")
    x = torch.zeros((0, 8, 3), device="cuda")
    assert op.matvec(x).shape == (0, 8, 2)
    with pytest.raises(TypeError):
        op.matvec(torch.zeros((8, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        op.matvec(torch.zeros((8, 4), device="cuda"))
    lib = btt.load()
    assert lib.btt_matvec_f64(op.handle, x.data_ptr(), x.data_ptr(), 1, None) == btt._lib.BTT_ERR_ARG
    y = torch.zeros((1, 8, 3), device="cuda")
    assert lib.btt_hessian(op.handle, y.data_ptr(), None, y.data_ptr(), 1, None) == btt._lib.BTT_ERR_ARG
    assert lib.btt_matvec(op.handle, y.data_ptr(), y.data_ptr(), -1, None) == btt._lib.BTT_ERR_ARG
    op.close()
    with pytest.raises(btt.BttError):
        btt.Operator(synth.blocks(synth.Workload("u", 11, 1, 1, tau=1.0)), precision="f32")
    with pytest.raises(btt.BttError) as e:
        btt.Operator(F, precision="f32", max_nrhs=4, workspace_limit=100)
    assert e.value.status == btt._lib.BTT_ERR_OOM


# ------------------------------------------------ long transforms (N_t sweep)
LONG = [  # (N_t, N_d, N_m, precision): fixed plans at 2*N_t = 4000, 8000; one column pair per CTA beyond 8192
    (2000, 3, 45, "f32"),      # fixed plan 8,4,5,5,5 with 4 columns per CTA, ragged tile
    (4000, 2, 17, "f32"),      # fixed plan 8,8,5,5,5 with 2 columns per CTA
    (2000, 3, 33, "f16s"),
    (5000, 3, 9, "f32"),       # setup transform in shared memory
    (10000, 2, 5, "f32"),      # setup transform in global scratch
    (12288, 1, 3, "f32"),      # longest transform
    (9000, 2, 5, "f16s"),      # global scratch with the per-frequency maxima
    (7000, 2, 3, "f64"),       # FP64 matvec transforms in 219 KB of shared memory
]


@pytest.mark.parametrize("case", LONG)
def test_long_transforms(case):
    """Against the oracle's FFT algorithm (pinned to the direct definition
    on the CPU), which is the only oracle fast enough at these N_t."""
    N_t, N_d, N_m, prec = case
    w = synth.Workload("long", N_t, N_d, N_m, tau=N_t / 5, seed=N_t)
    is64 = prec == "f64"
    F, m, d, g = inputs(w, nrhs=2, fp32=not is64)
    dt = torch.float64 if is64 else torch.float32
    Fh = fft_method.setup(F)
    tol = 1e-12 if is64 else TOL[prec]
    with btt.Operator(F, precision=prec, max_nrhs=2) as op:
        dm = host(op.matvec(dev(m, dt)))
        md = host(op.adjoint(dev(d, dt)))
        hm = host(op.hessian(dev(m, dt), dev(g, dt)))
        op.device_status()
    assert direct.rel_l2(dm, fft_method.forward(Fh, m)) < tol
    assert direct.rel_l2(md, fft_method.adjoint(Fh, d)) < tol
    assert direct.rel_l2(hm, fft_method.hessian(Fh, m, g)) < tol
    # a sampled entry of the plain definition as well
    t, s = N_t - 1, N_d - 1
    ref = sum(F[t - j, s] @ m[0, j] for j in range(N_t))
    assert abs(dm[0, t, s] - ref) <= 10 * tol * np.linalg.norm(dm[0]) / np.sqrt(dm[0].size) + 1e-12


@pytest.mark.parametrize("N_t", [2000, 6000])
def test_long_transform_tensor_path(N_t):
    w = synth.Workload("long-tc", N_t, 20, 40, tau=N_t / 5, seed=61)
    F, m, d, g = inputs(w, nrhs=2)
    Fh = fft_method.setup(F)
    with btt.Operator(F, precision="bf16", max_nrhs=2, gemm="tensor") as op:
        dm = host(op.matvec(dev(m, torch.float32)))
        md = host(op.adjoint(dev(d, torch.float32)))
        op.device_status()
    assert direct.rel_l2(dm, fft_method.forward(Fh, m)) < TOL["bf16"]
    assert direct.rel_l2(md, fft_method.adjoint(Fh, d)) < TOL["bf16"]


# ------------------------------------- single-vector F (one warp per row)
ROWS_SHAPES = [  # (N_t, N_d, N_m): 8- and 20-row CTAs, ragged rows, chunks of 2048 with tails
    (16, 7, 2500), (16, 13, 33), (16, 20, 1), (16, 41, 4097), (12, 100, 2048), (10, 3, 6000),
]


@pytest.mark.parametrize("shape", ROWS_SHAPES)
@pytest.mark.parametrize("prec", ["f32", "f16s", "bf16", "bf16x2", "fp8s"])
def test_single_vector_forward(shape, prec):
    N_t, N_d, N_m = shape
    w = synth.Workload("rows", N_t, N_d, N_m, tau=N_t / 3, envelope=prec != "f32", seed=N_d * 7 + N_m)
    F, m, _, _ = inputs(w, nrhs=1)
    with btt.Operator(F, precision=prec, max_nrhs=1) as op:
        got = host(op.matvec(dev(m, torch.float32)))
        op.device_status()
    assert direct.rel_l2(got, direct.forward(F, m)) < TOL[prec]
    if prec != "f32":
        # against the oracle's algorithm on the same rounded Fhat: only FP32 arithmetic remains
        Fq = quantize.quantize(fft_method.setup(F), QFMT[prec])
        assert direct.rel_l2(got, fft_method.forward(Fq, m)) < 4e-6
