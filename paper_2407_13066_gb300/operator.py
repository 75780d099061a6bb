"""Operator handle over the C ABI (argument marshalling only)."""
import ctypes

import numpy as np

from . import _lib


def _torch():
    import torch
    return torch


def _ptr_and_stream(x, stream):
    """(pointer, stream handle) for a torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data, stream
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch.Tensor or numpy.ndarray, got %r" % type(x))
    if not x.is_contiguous():
        raise ValueError("tensors must be contiguous")
    if stream is None and x.is_cuda:
        stream = torch.cuda.current_stream(x.device).cuda_stream
    return x.data_ptr(), stream


class Operator:
    """One block lower-triangular Toeplitz operator resident on the GPU.

    blocks: float64 [N_t][N_d][N_m] first block column (torch tensor on any
    device, or numpy array).  precision: 'f32', 'f16s', 'bf16', 'bf16x2',
    'fp8s' or 'f64'.  max_nrhs: right-hand sides one internal pass holds.
    """

    def __init__(self, blocks, precision="f32", max_nrhs=1, workspace_limit=0, stream=None, gemm="auto",
                 host_staging=-1):
        lib = _lib.load()
        if blocks.dtype not in (np.float64,) and str(blocks.dtype) != "torch.float64":
            raise TypeError("blocks must be float64")
        N_t, N_d, N_m = (int(v) for v in blocks.shape)
        ptr, st = _ptr_and_stream(blocks, stream)
        opt = _lib.BttOptions()
        lib.btt_default_options(ctypes.byref(opt))
        opt.precision = _lib.PRECISIONS[precision]
        opt.max_nrhs = int(max_nrhs)
        opt.workspace_limit = int(workspace_limit)
        opt.stream = st
        opt.gemm = _lib.GEMM_MODES[gemm]
        opt.host_staging = int(host_staging)
        h = ctypes.c_void_p()
        _lib.check(lib.btt_create(ctypes.byref(h), ptr, N_t, N_d, N_m, ctypes.byref(opt)))
        self._h = h
        self._lib = lib
        self.N_t, self.N_d, self.N_m = N_t, N_d, N_m
        self.precision = precision
        self.max_nrhs = int(max_nrhs)

    # -------------------------------------------------------------- utils
    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("operator is closed")
        return self._h

    @property
    def is64(self):
        return self.precision == "f64"

    def operator_bytes(self):
        return self._lib.btt_operator_bytes(self.handle)

    def workspace_bytes(self, nrhs=0):
        """Device workspace of this operator (nrhs <= 0), or of the same
        operator created with max_nrhs = nrhs."""
        return self._lib.btt_workspace_bytes(self.handle, int(nrhs))

    def fhat_ld(self):
        return self._lib.btt_fhat_ld(self.handle)

    def copy_fhat(self):
        """Stored Fhat as raw bytes (numpy uint8) and the per-frequency scales."""
        nbytes = self.operator_bytes() - (4 * (self.N_t + 1) if self.precision in ("f16s", "fp8s") else 0)
        raw = np.empty(nbytes, dtype=np.uint8)
        sc = np.empty(self.N_t + 1, dtype=np.float32)
        _lib.check(self._lib.btt_copy_fhat(self.handle, raw.ctypes.data, sc.ctypes.data))
        return raw, sc

    def device_status(self, stream=None):
        """Synchronise and raise if a bounded device wait of this operator ran out."""
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        _lib.check(self._lib.btt_device_status(self.handle, stream))

    def profile(self, on=True):
        """Enable (and reset) or disable the library's per-stage event timers."""
        _lib.check(self._lib.btt_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self):
        """{stage: (milliseconds, launches)} since the last reset."""
        ms = (ctypes.c_double * 5)()
        n = (ctypes.c_longlong * 5)()
        _lib.check(self._lib.btt_profile_read(self.handle, ms, n))
        return {name: (ms[i], n[i]) for i, name in enumerate(_lib.STAGES)}

    def save(self, path):
        """Writes the stored Fhat (and scales) to an operator file."""
        _lib.check(self._lib.btt_save(self.handle, str(path).encode()))

    @classmethod
    def load(cls, path, max_nrhs=1, workspace_limit=0, stream=None, gemm="auto", host_staging=-1):
        """An operator from a file written by save(), without the setup
        transform; the storage format is the file's."""
        lib = _lib.load()
        opt = _lib.BttOptions()
        lib.btt_default_options(ctypes.byref(opt))
        opt.max_nrhs = int(max_nrhs)
        opt.workspace_limit = int(workspace_limit)
        opt.stream = stream
        opt.gemm = _lib.GEMM_MODES[gemm]
        opt.host_staging = int(host_staging)
        h = ctypes.c_void_p()
        _lib.check(lib.btt_load(ctypes.byref(h), str(path).encode(), ctypes.byref(opt)))
        self = cls.__new__(cls)
        self._h = h
        self._lib = lib
        N_t, N_d, N_m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(lib.btt_operator_shape(h, ctypes.byref(N_t), ctypes.byref(N_d), ctypes.byref(N_m)))
        self.N_t, self.N_d, self.N_m = N_t.value, N_d.value, N_m.value
        inv = {v: k for k, v in _lib.PRECISIONS.items()}
        self.precision = inv[lib.btt_precision_of(h)]
        self.max_nrhs = int(max_nrhs)
        return self

    def close(self):
        if self._h is not None:
            self._lib.btt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ actions
    def _alloc_like(self, x, shape):
        if isinstance(x, np.ndarray):
            return np.empty(shape, dtype=x.dtype)
        return _torch().empty(shape, dtype=x.dtype, device=x.device)

    def _nrhs(self, x, n_space):
        if x.ndim == 2:
            if tuple(x.shape) != (self.N_t, n_space):
                raise ValueError("expected shape (%d, %d), got %s" % (self.N_t, n_space, tuple(x.shape)))
            return 1, ()
        if x.ndim == 3 and tuple(x.shape[1:]) == (self.N_t, n_space):
            return int(x.shape[0]), (int(x.shape[0]),)
        raise ValueError("expected shape ([nrhs,] %d, %d), got %s" % (self.N_t, n_space, tuple(x.shape)))

    def _check_dtype(self, x):
        want = "float64" if self.is64 else "float32"
        if str(x.dtype).replace("torch.", "") != want:
            raise TypeError("vectors of a %s operator must be %s" % (self.precision, want))

    def _call(self, name, x, n_in, n_out, out, stream, extra=None):
        self._check_dtype(x)
        nrhs, lead = self._nrhs(x, n_in)
        if out is None:
            out = self._alloc_like(x, lead + (self.N_t, n_out))
        else:
            self._check_dtype(out)
            if tuple(out.shape) != lead + (self.N_t, n_out):
                raise ValueError("output has shape %s" % (tuple(out.shape),))
        px, st = _ptr_and_stream(x, stream)
        po, _ = _ptr_and_stream(out, st)
        fn = getattr(self._lib, name + ("_f64" if self.is64 else ""))
        if extra is None:
            _lib.check(fn(self.handle, px, po, nrhs, st))
        else:
            pg = None
            if extra is not False:
                self._check_dtype(extra)
                if tuple(extra.shape) != (self.N_t, self.N_d):
                    raise ValueError("gamma_inv must have shape (%d, %d)" % (self.N_t, self.N_d))
                pg, _ = _ptr_and_stream(extra, st)
            _lib.check(fn(self.handle, px, pg, po, nrhs, st))
        return out

    def cg(self, b, alpha, gamma_inv=None, x0=None, max_iter=200, tol=1e-6, stream=None):
        """Solve (F* Gamma^-1 F + alpha I) x = b by conjugate gradients on the
        device (btt_cg).  b: CUDA float32 [nrhs][N_t][N_m] or [N_t][N_m].
        Returns (x, iterations, relative residuals)."""
        import torch
        if self.is64:
            raise TypeError("btt_cg needs an FP32 operator")
        if not (isinstance(b, torch.Tensor) and b.is_cuda):
            raise TypeError("b must be a CUDA tensor")
        nrhs, lead = self._nrhs(b, self.N_m)
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        its = (ctypes.c_int * max(1, nrhs))()
        rel = (ctypes.c_float * max(1, nrhs))()
        pb, st = _ptr_and_stream(b.contiguous(), stream)
        pg = None
        if gamma_inv is not None:
            self._check_dtype(gamma_inv)
            pg, _ = _ptr_and_stream(gamma_inv, st)
        _lib.check(self._lib.btt_cg(self.handle, pb, pg, float(alpha), x.data_ptr(), nrhs, int(max_iter),
                                    float(tol), its, rel, st))
        return x, list(its)[:nrhs], list(rel)[:nrhs]

    def matvec(self, m, out=None, stream=None):
        """d = F m; m [nrhs][N_t][N_m] or [N_t][N_m]."""
        return self._call("btt_matvec", m, self.N_m, self.N_d, out, stream)

    def adjoint(self, d, out=None, stream=None, gamma_inv=None):
        """m = F* d; d [nrhs][N_t][N_d] or [N_t][N_d].  With gamma_inv
        [N_t][N_d]: m = F* (Gamma^-1 d) (btt_adjoint_weighted, FP32 operators),
        the second pass of a Hessian split over GPUs."""
        if gamma_inv is None:
            return self._call("btt_adjoint", d, self.N_d, self.N_m, out, stream)
        if self.is64:
            raise TypeError("btt_adjoint_weighted needs an FP32 operator")
        return self._call("btt_adjoint_weighted", d, self.N_d, self.N_m, out, stream, extra=gamma_inv)

    def hessian(self, m, gamma_inv=None, out=None, stream=None):
        """y = F* Gamma^-1 F m; gamma_inv [N_t][N_d] or None (identity)."""
        return self._call("btt_hessian", m, self.N_m, self.N_m, out, stream,
                          extra=False if gamma_inv is None else gamma_inv)
