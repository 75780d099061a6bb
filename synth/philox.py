"""NumPy implementation of the seeded input generator (see ``philox.h``).

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) written out over uint64
arrays, with the same counter/key layout and the same Box-Muller mapping as
the C and CUDA builds.  It is slow but obviously direct; the tests use it to
check the compiled builds word for word.
"""
import numpy as np

_M32 = np.uint64(0xFFFFFFFF)
_MUL0 = np.uint64(0xD2511F53)
_MUL1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on arrays (or scalars) of 32-bit words held in uint64."""
    c = [np.asarray(x, dtype=np.uint64) & _M32 for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint64) & _M32
    k1 = np.asarray(k1, dtype=np.uint64) & _M32
    for _ in range(10):
        p0 = _MUL0 * c[0]
        p1 = _MUL1 * c[2]
        c = [(p1 >> _S32) ^ c[1] ^ k0, p1 & _M32, (p0 >> _S32) ^ c[3] ^ k1, p0 & _M32]
        k0 = (k0 + _W0) & _M32
        k1 = (k1 + _W1) & _M32
    return c


def _words(seed, tensor_id, e):
    e = np.asarray(e, dtype=np.uint64)
    j = e >> np.uint64(1)
    seed = np.uint64(seed)
    return philox4x32_10(j & _M32, j >> _S32, np.uint64(tensor_id), 0, seed & _M32, seed >> _S32)


def _u53(a, b):
    m = (a << np.uint64(21)) | (b >> np.uint64(11))
    return (m.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed, tensor_id, e):
    """Standard normal for element indices ``e`` of stream (seed, tensor_id)."""
    e = np.asarray(e, dtype=np.uint64)
    w = _words(seed, tensor_id, e)
    u1 = _u53(w[0], w[1])
    u2 = _u53(w[2], w[3])
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 6.283185307179586476925286766559 * u2
    odd = (e & np.uint64(1)).astype(bool)
    return np.where(odd, rad * np.sin(ang), rad * np.cos(ang))


def uniform(seed, tensor_id, e):
    """Uniform in (0,1) for element indices ``e`` of stream (seed, tensor_id)."""
    e = np.asarray(e, dtype=np.uint64)
    w = _words(seed, tensor_id, e)
    odd = (e & np.uint64(1)).astype(bool)
    return np.where(odd, _u53(w[2], w[3]), _u53(w[0], w[1]))


def block_entries(seed, N_d, N_m, tau, env_d, env_m, k, s, l):
    """F_k[s][l] of the synthetic first block column (see ``philox.h``)."""
    k = np.asarray(k, dtype=np.int64)
    s = np.asarray(s, dtype=np.int64)
    l = np.asarray(l, dtype=np.int64)
    v = normal(seed, 0, ((k * N_d + s) * N_m + l).astype(np.uint64))
    if tau > 0:
        v = v * np.exp(-k.astype(np.float64) / tau)
    if env_d is not None:
        v = v * np.asarray(env_d)[s]
    if env_m is not None:
        v = v * np.asarray(env_m)[l]
    return v
