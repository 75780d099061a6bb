"""Reduced-precision storage of F-hat as plain element maps (FP64 in/out).

TEST INFRASTRUCTURE ONLY.  The paper stores F-hat in complex128 only; the
reduced storage formats below are the readings used by the library:

  fp32      x32 = round-to-nearest FP32 of each real/imaginary part.
  fp16s     per frequency w: s_w = fp32(max_{s,l} max(|Re|,|Im|) / 2^14)
            (s_w = 1 for an all-zero slice); code = fp16(fp32(x / s_w));
            value = code * s_w.
  bf16      code = bf16(fp32(x)), round to nearest even at each step.
  bf16x2    hi = bf16(fp32(x)); lo = bf16(fp32(x - hi)); value = hi + lo.
  fp8s      per frequency w: s_w = fp32(max_{s,l} max(|Re|,|Im|) / 256)
            (1 for an all-zero slice); code = e4m3(fp32(x / s_w)) (nearest
            even, saturating at 448); value = code * s_w.
"""
import numpy as np


def to_bf16(x):
    """Round float64 -> float32 -> bfloat16 (nearest even); returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    # round to nearest even on the low 16 bits (finite inputs)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def to_e4m3(x):
    """Round to FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa
    bits; subnormal spacing 2^-9; largest finite 448), nearest even,
    saturating; returned as float64."""
    f = np.asarray(x, dtype=np.float64)
    a = np.abs(f)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    step = 2.0 ** (e - 3)
    q = np.minimum(np.round(a / step) * step, 448.0)
    return np.where(f < 0, -q, q)


def _parts(z):
    z = np.asarray(z)
    return z.real.astype(np.float64), z.imag.astype(np.float64)


def fp16_scales(Fhat, target=16384.0):
    """Per-frequency scale s_w (float64 holding an FP32 value)."""
    re, im = _parts(Fhat)
    mx = np.maximum(np.abs(re), np.abs(im)).reshape(Fhat.shape[0], -1).max(axis=1)
    s = (mx / target).astype(np.float32).astype(np.float64)
    s[mx == 0] = 1.0
    return s


def fp8_scales(Fhat):
    return fp16_scales(Fhat, 256.0)


def quantize(Fhat, fmt):
    """Value of F-hat after storage in ``fmt`` (complex128)."""
    re, im = _parts(Fhat)
    if fmt == "fp32":
        q = lambda v: v.astype(np.float32).astype(np.float64)
    elif fmt == "fp16s":
        s = fp16_scales(Fhat).reshape((-1,) + (1,) * (Fhat.ndim - 1))
        q = lambda v: (v / s).astype(np.float32).astype(np.float16).astype(np.float64) * s
    elif fmt == "bf16":
        q = to_bf16
    elif fmt == "fp8s":
        s = fp8_scales(Fhat).reshape((-1,) + (1,) * (Fhat.ndim - 1))
        q = lambda v: to_e4m3((v / s).astype(np.float32).astype(np.float64)) * s
    elif fmt == "bf16x2":
        def q(v):
            hi = to_bf16(v)
            return hi + to_bf16(v - hi)
    else:
        raise ValueError(fmt)
    return q(re) + 1j * q(im)
