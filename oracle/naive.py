"""ctypes wrapper of naive.c (TEST INFRASTRUCTURE ONLY)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle_naive.so")
_lib = None


def build(force=False):
    src = os.path.join(_HERE, "naive.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", _SO, src])


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        for f in (lib.oracle_naive_forward, lib.oracle_naive_adjoint):
            f.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3
            f.restype = None
        _lib = lib
    return _lib


def forward(F, m):
    F = np.ascontiguousarray(F, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    N_t, N_d, N_m = F.shape
    d = np.empty((N_t, N_d), dtype=np.float64)
    _load().oracle_naive_forward(N_t, N_d, N_m, F.ctypes.data, m.ctypes.data, d.ctypes.data)
    return d


def adjoint(F, d):
    F = np.ascontiguousarray(F, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    N_t, N_d, N_m = F.shape
    m = np.empty((N_t, N_m), dtype=np.float64)
    _load().oracle_naive_adjoint(N_t, N_d, N_m, F.ctypes.data, d.ctypes.data, m.ctypes.data)
    return m
