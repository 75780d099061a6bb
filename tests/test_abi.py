"""The C-ABI library builds, loads and exports every declared symbol; host
argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(btt_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = btt.load()
    decl = declared_functions()
    assert len(decl) >= 17
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTS) == sorted(n for n in decl if n in _lib.EXPORTS)
    assert set(decl) <= set(_lib.EXPORTS) | set(getattr(_lib, "EXTRA_EXPORTS", []))


def test_exports_in_dynamic_symbol_table():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", btt.library_path()], capture_output=True,
                         text=True).stdout
    syms = set(re.findall(r"\b(btt_[a-z0-9_]+)\b", out))
    assert set(declared_functions()) <= syms
    # nothing but the C ABI is exported
    assert not re.search(r"\bT _Z", out)


def test_host_only_calls():
    lib = btt.load()
    assert lib.btt_version().startswith(b"btt")
    assert [lib.btt_entry_bytes(p) for p in range(5)] == [8, 4, 4, 8, 16]
    assert lib.btt_entry_bytes(9) == 0
    opt = _lib.BttOptions()
    lib.btt_default_options(ctypes.byref(opt))
    assert (opt.precision, opt.max_nrhs, opt.workspace_limit, opt.stream) == (0, 1, 0, None)


def test_argument_errors_without_gpu():
    lib = btt.load()
    assert lib.btt_create(None, None, 4, 4, 4, None) == _lib.BTT_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.btt_create(ctypes.byref(h), None, 4, 4, 4, None) == _lib.BTT_ERR_ARG
    assert b"null blocks" in lib.btt_last_error()
    buf = (ctypes.c_double * 8)()
    assert lib.btt_create(ctypes.byref(h), buf, 0, 4, 4, None) == _lib.BTT_ERR_ARG
    assert lib.btt_matvec(None, buf, buf, 1, None) == _lib.BTT_ERR_ARG
    assert lib.btt_destroy(None) == _lib.BTT_OK
    assert lib.btt_operator_bytes(None) == 0


def test_unsupported_lengths_rejected_on_host():
    lib = btt.load()
    h = ctypes.c_void_p()
    buf = (ctypes.c_double * 64)()
    for N_t in (11, 13, 4097):   # 2*N_t has a prime factor > 7
        opt = _lib.BttOptions()
        lib.btt_default_options(ctypes.byref(opt))
        assert lib.btt_create(ctypes.byref(h), buf, N_t, 1, 1, ctypes.byref(opt)) == _lib.BTT_ERR_UNSUPPORTED
    big = np.zeros(12500, dtype=np.float64)
    opt = _lib.BttOptions()
    lib.btt_default_options(ctypes.byref(opt))
    # 2*N_t = 25000 = 2^3 5^5 factors, but exceeds the longest transform (24576)
    assert lib.btt_create(ctypes.byref(h), big.ctypes.data, 12500, 1, 1, ctypes.byref(opt)) == _lib.BTT_ERR_UNSUPPORTED
    assert b"24576" in lib.btt_last_error()
    # FP64 storage keeps its transforms in shared memory: 2*N_t = 15000 is too long
    opt.precision = _lib.PRECISIONS["f64"]
    assert lib.btt_create(ctypes.byref(h), big.ctypes.data, 7500, 1, 1, ctypes.byref(opt)) == _lib.BTT_ERR_UNSUPPORTED
    assert b"FP64" in lib.btt_last_error()


def test_operator_files_rejected_on_host(tmp_path):
    """btt_load answers a missing, foreign or inconsistent file before any
    device work."""
    lib = btt.load()
    h = ctypes.c_void_p()
    assert lib.btt_load(ctypes.byref(h), str(tmp_path / "missing").encode(), None) == _lib.BTT_ERR_ARG
    bad = tmp_path / "bad"
    bad.write_bytes(b"not an operator file" * 8)
    assert lib.btt_load(ctypes.byref(h), str(bad).encode(), None) == _lib.BTT_ERR_ARG
    assert b"not an operator file" in lib.btt_last_error()
    # a well-formed header whose byte count does not match its sizes
    import struct
    hdr = b"BTTFHAT1" + struct.pack("<6i", 1, 0, 4, 2, 3, 4) + struct.pack("<2Q", 999, 0) + bytes(32)
    assert len(hdr) == 80
    inc = tmp_path / "inconsistent"
    inc.write_bytes(hdr)
    assert lib.btt_load(ctypes.byref(h), str(inc).encode(), None) == _lib.BTT_ERR_ARG
    assert b"inconsistent" in lib.btt_last_error()
    assert not h.value


def test_fault_injection_arguments():
    lib = btt.load()
    assert lib.btt_inject_fault(7, 1) == _lib.BTT_ERR_ARG
    assert lib.btt_inject_fault(_lib.FAULTS["alloc"], -1) == _lib.BTT_ERR_ARG
    assert lib.btt_inject_fault(_lib.FAULTS["launch"], 2) == _lib.BTT_OK
    assert lib.btt_inject_fault(_lib.FAULTS["none"], 0) == _lib.BTT_OK


def test_bounds_check_build_compiles():
    """The bounds-check build (-DBTT_CHECK) compiles and exports the same ABI,
    and reports itself as such; the normal build does not."""
    from paper_2407_13066_gb300 import build
    path = build.build(check=True)
    chk = ctypes.CDLL(path)
    assert chk.btt_check_build() == 1
    for name in declared_functions():
        assert hasattr(chk, name), name
    assert btt.load().btt_check_build() == (1 if _lib.check_build_requested() else 0)
