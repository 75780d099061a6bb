"""ctypes binding of libbtt.so (include/btt.h): argument marshalling only.

Every step of every action runs in the library's CUDA kernels; there is no
other implementation behind these names.  If the library cannot be loaded
the calls raise -- nothing falls back to the CPU.
"""
import ctypes
import os

from . import build as _build

BTT_OK, BTT_ERR_ARG, BTT_ERR_OOM, BTT_ERR_CUDA, BTT_ERR_TIMEOUT, BTT_ERR_UNSUPPORTED = range(6)
PRECISIONS = {"f32": 0, "f16s": 1, "bf16": 2, "bf16x2": 3, "f64": 4, "fp8s": 5}
STATUS_NAMES = {0: "BTT_OK", 1: "BTT_ERR_ARG", 2: "BTT_ERR_OOM", 3: "BTT_ERR_CUDA",
                4: "BTT_ERR_TIMEOUT", 5: "BTT_ERR_UNSUPPORTED"}

# every symbol include/btt.h declares, in declaration order
EXPORTS = ["btt_default_options", "btt_create", "btt_destroy", "btt_matvec", "btt_adjoint",
           "btt_adjoint_weighted", "btt_hessian", "btt_hessian_batched", "btt_cg", "btt_matvec_f64", "btt_adjoint_f64", "btt_hessian_f64",
           "btt_precision_of", "btt_operator_shape", "btt_operator_bytes", "btt_workspace_bytes", "btt_entry_bytes",
           "btt_copy_fhat", "btt_fhat_ld", "btt_save", "btt_load", "btt_inject_fault", "btt_profile_enable", "btt_profile_read",
           "btt_matvec_noalloc", "btt_device_status", "btt_check_build", "btt_check_status", "btt_check_selftest",
           "btt_selftest_wait", "btt_server_create", "btt_server_submit",
           "btt_server_wait", "btt_server_poll", "btt_server_stats", "btt_server_inject",
           "btt_server_destroy", "btt_launch_count", "btt_last_error", "btt_version"]
GEMM_MODES = {"auto": 0, "simt": 1, "tensor": 2}
FAULTS = {"none": 0, "alloc": 1, "launch": 2}
STAGES = ["rfft", "gemv_f", "mid", "gemv_adj", "irfft"]


class BttOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("workspace_limit", ctypes.c_size_t), ("stream", ctypes.c_void_p),
                ("gemm", ctypes.c_int), ("host_staging", ctypes.c_int)]


class ServingStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("vectors_completed", ctypes.c_longlong),
                ("batches", ctypes.c_longlong), ("mean_batch_vectors", ctypes.c_double),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_mean_ms", ctypes.c_double), ("span_s", ctypes.c_double),
                ("pool_bytes", ctypes.c_size_t), ("pool_in_use", ctypes.c_size_t),
                ("pool_high_water", ctypes.c_size_t), ("waiting", ctypes.c_longlong),
                ("admitted", ctypes.c_longlong), ("running", ctypes.c_longlong)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class BttError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def check_build_requested():
    """True when the environment asks for the bounds-check build (BTT_CHECK=1)."""
    return os.environ.get("BTT_CHECK", "0") not in ("", "0")


def library_path():
    return _build.lib_path(check_build_requested())


def load(build_if_missing=True):
    """Loads libbtt.so, or libbtt_check.so when BTT_CHECK=1 (building it in-tree
    first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    check = check_build_requested()
    if build_if_missing:
        _build.build(check=check)
    path = _build.lib_path(check)
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run paper_2407_13066_gb300.build.build(check=%s)"
                           % (path, check))
    lib = ctypes.CDLL(path)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    sig = {
        "btt_default_options": ([ctypes.POINTER(BttOptions)], None),
        "btt_create": ([ctypes.POINTER(vp), vp, i, i, i, ctypes.POINTER(BttOptions)], i),
        "btt_destroy": ([vp], i),
        "btt_matvec": ([vp, vp, vp, i, vp], i),
        "btt_adjoint": ([vp, vp, vp, i, vp], i),
        "btt_adjoint_weighted": ([vp, vp, vp, vp, i, vp], i),
        "btt_check_build": ([], i),
        "btt_check_status": ([vp], i),
        "btt_check_selftest": ([vp], i),
        "btt_hessian": ([vp, vp, vp, vp, i, vp], i),
        "btt_hessian_batched": ([vp, vp, vp, vp, i, vp], i),
        "btt_cg": ([vp, vp, vp, ctypes.c_float, vp, i, i, ctypes.c_float, vp, vp, vp], i),
        "btt_matvec_f64": ([vp, vp, vp, i, vp], i),
        "btt_adjoint_f64": ([vp, vp, vp, i, vp], i),
        "btt_hessian_f64": ([vp, vp, vp, vp, i, vp], i),
        "btt_precision_of": ([vp], i),
        "btt_operator_shape": ([vp, vp, vp, vp], i),
        "btt_server_create": ([ctypes.POINTER(vp), vp, vp, i, sz, i], i),
        "btt_server_submit": ([vp, i, vp, vp, i, ctypes.POINTER(ctypes.c_longlong)], i),
        "btt_server_wait": ([vp, ctypes.c_longlong, ctypes.c_double], i),
        "btt_server_poll": ([vp, ctypes.c_longlong, ctypes.POINTER(i)], i),
        "btt_server_stats": ([vp, ctypes.POINTER(ServingStats), i], i),
        "btt_server_inject": ([vp, i], i),
        "btt_server_destroy": ([vp], i),
        "btt_operator_bytes": ([vp], sz),
        "btt_workspace_bytes": ([vp, i], sz),
        "btt_entry_bytes": ([i], sz),
        "btt_copy_fhat": ([vp, vp, vp], i),
        "btt_fhat_ld": ([vp], i),
        "btt_save": ([vp, ctypes.c_char_p], i),
        "btt_load": ([ctypes.POINTER(vp), ctypes.c_char_p, ctypes.POINTER(BttOptions)], i),
        "btt_inject_fault": ([i, i], i),
        "btt_profile_enable": ([vp, i], i),
        "btt_profile_read": ([vp, vp, vp], i),
        "btt_matvec_noalloc": ([vp, i, i, i, vp, vp, i, vp], i),
        "btt_device_status": ([vp, vp], i),
        "btt_selftest_wait": ([vp, ctypes.c_double, vp], i),
        "btt_launch_count": ([], ctypes.c_longlong),
        "btt_last_error": ([], ctypes.c_char_p),
        "btt_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def check(status):
    if status != BTT_OK:
        raise BttError(status, load().btt_last_error().decode())
