"""Workload recipes and the compiled generator builds.

Every workload is synthetic, drawn from the counter-based generator keyed by
(seed, tensor id, element index), so any entry of any input can be drawn on
its own -- the oracle draws only the block rows it needs, the GPU side fills
whole tensors on the device.
"""
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import philox as _np_philox

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libsynth_host.so")
_DEV_SO = os.path.join(_HERE, "libsynth_dev.so")

T_BLOCKS, T_PARAM, T_DATA, T_NOISE, T_ENV_D, T_ARRIVAL, T_ENV_M, T_DIRS, T_WEIGHTS = range(9)


@dataclass(frozen=True)
class Workload:
    """One block lower-triangular Toeplitz operator and its inputs.

    Blocks: F_k[s][l] = N(0,1) * exp(-k/tau) * env_d[s] * env_m[l]
    (tau <= 0: no decay; envelope False: env = 1).
    """
    name: str
    N_t: int
    N_d: int
    N_m: int
    tau: float
    envelope: bool = False
    nrhs: int = 1
    seed: int = 0

    @property
    def n_freq(self):
        return self.N_t + 1

    def fhat_bytes(self, bytes_per_entry=8):
        return self.n_freq * self.N_d * self.N_m * bytes_per_entry


WORKLOADS = {
    # F and F* in FP64 on a small operator, checked against a dense matrix.
    "fp64-small": Workload("fp64-small", 64, 8, 32, tau=16.0),
    # single-vector bandwidth path, complex64 F-hat of 8.0 GB.
    "bandwidth": Workload("bandwidth", 1000, 100, 10000, tau=200.0),
    # storage-precision sweep, blocks shaped by a smooth spatial envelope.
    "precision": Workload("precision", 512, 600, 20000, tau=0.0, envelope=True),
    # the bandwidth operator with a tenth of the parameters (Fhat 0.8 GB,
    # still far above L2): small enough for multi-pass profiler captures.
    "bandwidth-small": Workload("bandwidth-small", 1000, 100, 1000, tau=200.0),
    # the bandwidth operator's rows (N_m = 10 000) over a tenth of the
    # frequencies (Fhat 0.8 GB): per-CTA work as at full size, for profiling.
    "bandwidth-rows": Workload("bandwidth-rows", 100, 100, 10000, tau=20.0),
    # 64 right-hand sides at once.
    "multi-rhs": Workload("multi-rhs", 256, 200, 50000, tau=64.0, nrhs=64),
}

# the multi-rhs operator with a tenth of the parameters (BF16 Fhat 1.0 GB),
# for profiler captures of the multi-right-hand-side kernels.
WORKLOADS["multi-rhs-small"] = Workload("multi-rhs-small", 256, 200, 5000, tau=64.0, nrhs=64)
# the serving workload's largest operator with a tenth of the parameters
# (BF16 Fhat 2.05 GB), 32 vectors: profiler captures at 2 N_t = 2048
WORKLOADS["serve-3-small"] = Workload("serve-3-small", 1024, 100, 5000, tau=1024 / 5, nrhs=32)

# four resident operators of the serving workload, decay tau = N_t / 5
SERVING_OPERATORS = [
    Workload("serve-0", 128, 50, 2000, tau=128 / 5, seed=10),
    Workload("serve-1", 256, 200, 10000, tau=256 / 5, seed=11),
    Workload("serve-2", 512, 600, 20000, tau=512 / 5, seed=12),
    Workload("serve-3", 1024, 100, 50000, tau=1024 / 5, seed=13),
]


# ----------------------------------------------------------------- builds
def build(device=True, force=False):
    """Compile the host build (gcc) and, if asked, the device build (nvcc)."""
    src = os.path.join(_HERE, "synth_host.c")
    if force or not os.path.exists(_HOST_SO) or os.path.getmtime(_HOST_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               "-o", _HOST_SO, src, "-lm"])
    if device:
        src = os.path.join(_HERE, "synth_dev.cu")
        if force or not os.path.exists(_DEV_SO) or os.path.getmtime(_DEV_SO) < os.path.getmtime(src):
            subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                                   "-Xcompiler", "-fPIC", "-shared", "-o", _DEV_SO, src])


_host = None
_dev = None


def host_lib():
    global _host
    if _host is None:
        build(device=False)
        lib = ctypes.CDLL(_HOST_SO)
        u64, u32, i64, dp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
        lib.synth_host_philox.argtypes = [u32] * 6 + [dp]
        lib.synth_host_normal.argtypes = [u64, u32, u64, i64, dp]
        lib.synth_host_uniform.argtypes = [u64, u32, u64, i64, ctypes.c_double, ctypes.c_double, dp]
        lib.synth_host_blocks.argtypes = [u64, i64, i64, ctypes.c_double, dp, dp, i64, i64, dp]
        lib.synth_host_block_entries.argtypes = [u64, i64, i64, ctypes.c_double, dp, dp, i64,
                                                 dp, dp, dp, dp]
        for f in ("synth_host_philox", "synth_host_normal", "synth_host_uniform",
                  "synth_host_blocks", "synth_host_block_entries"):
            getattr(lib, f).restype = None
        _host = lib
    return _host


def dev_lib():
    global _dev
    if _dev is None:
        build(device=True)
        lib = ctypes.CDLL(_DEV_SO)
        u64, u32, i64, dp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
        lib.synth_dev_normal.argtypes = [u64, u32, u64, i64, dp, dp, dp]
        lib.synth_dev_uniform.argtypes = [u64, u32, u64, i64, ctypes.c_double, ctypes.c_double,
                                          dp, dp, dp]
        lib.synth_dev_blocks.argtypes = [u64, i64, i64, ctypes.c_double, dp, dp, i64, i64, dp, dp]
        for f in ("synth_dev_normal", "synth_dev_uniform", "synth_dev_blocks"):
            getattr(lib, f).restype = ctypes.c_int
        _dev = lib
    return _dev


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- drawing
def envelope(w: Workload, side: str):
    """Smooth random spatial envelope in [0.1, 1] over the data ('d') or
    parameter ('m') index: 0.1 + 0.9*(1/2 + 1/2*S(x)/sum|a_q|) with
    S(x) = sum_{q=1..3} a_q cos(2*pi*q*x + phi_q), x = index/length,
    a_q uniform in (-1,1), phi_q uniform in (0, 2*pi).  The product of the
    two sides lies in [0.01, 1].  None when the workload has no envelope."""
    if not w.envelope:
        return None
    n = w.N_d if side == "d" else w.N_m
    tid = T_ENV_D if side == "d" else T_ENV_M
    u = _np_philox.uniform(w.seed, tid, np.arange(6, dtype=np.uint64))
    a = 2.0 * u[:3] - 1.0
    phi = 2.0 * np.pi * u[3:]
    x = np.arange(n, dtype=np.float64) / n
    q = np.arange(1, 4, dtype=np.float64)
    S = (a[:, None] * np.cos(2.0 * np.pi * q[:, None] * x[None, :] + phi[:, None])).sum(0)
    return 0.1 + 0.9 * (0.5 + 0.5 * S / np.abs(a).sum())


def normals(seed, tensor_id, count, start=0):
    out = np.empty(int(count), dtype=np.float64)
    host_lib().synth_host_normal(seed, tensor_id, start, int(count), _ptr(out))
    return out


def uniforms(seed, tensor_id, count, lo=0.0, hi=1.0, start=0):
    out = np.empty(int(count), dtype=np.float64)
    host_lib().synth_host_uniform(seed, tensor_id, start, int(count), lo, hi, _ptr(out))
    return out


def blocks(w: Workload, k0=0, k1=None):
    """Blocks F_k, k in [k0, k1), as a float64 array [k1-k0][N_d][N_m]."""
    k1 = w.N_t if k1 is None else k1
    out = np.empty((k1 - k0, w.N_d, w.N_m), dtype=np.float64)
    ed, em = envelope(w, "d"), envelope(w, "m")
    host_lib().synth_host_blocks(w.seed, w.N_d, w.N_m, float(w.tau), _ptr(ed), _ptr(em),
                                 k0, k1, _ptr(out))
    return out


def block_entries(w: Workload, k, s, l):
    """Scattered entries F_k[s][l] (broadcast index arrays)."""
    k, s, l = np.broadcast_arrays(np.asarray(k, np.int64), np.asarray(s, np.int64),
                                  np.asarray(l, np.int64))
    shape = k.shape
    k, s, l = (np.ascontiguousarray(a.ravel()) for a in (k, s, l))
    out = np.empty(k.size, dtype=np.float64)
    ed, em = envelope(w, "d"), envelope(w, "m")
    host_lib().synth_host_block_entries(w.seed, w.N_d, w.N_m, float(w.tau), _ptr(ed), _ptr(em),
                                        k.size, _ptr(k), _ptr(s), _ptr(l), _ptr(out))
    return out.reshape(shape)


def vectors(w: Workload, kind: str, nrhs=None, tensor_id=None):
    """nrhs N(0,1) vectors in time-outer layout: [nrhs][N_t][N_m] for kind
    'm', [nrhs][N_t][N_d] for kind 'd' (float64)."""
    nrhs = w.nrhs if nrhs is None else nrhs
    n = w.N_m if kind == "m" else w.N_d
    tid = tensor_id if tensor_id is not None else (T_PARAM if kind == "m" else T_DATA)
    return normals(w.seed, tid, nrhs * w.N_t * n).reshape(nrhs, w.N_t, n)


def noise_gamma_inv(w: Workload):
    """Diagonal noise precision: one variance sigma^2 ~ U[0.5, 2] per data
    entry (t, s); returns 1/sigma^2 as float64 [N_t][N_d]."""
    var = uniforms(w.seed, T_NOISE, w.N_t * w.N_d, 0.5, 2.0)
    return (1.0 / var).reshape(w.N_t, w.N_d)
