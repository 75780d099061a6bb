"""Serving of Hessian actions over resident operators (argument marshalling
over the library's native scheduler, btt_server_* in include/btt.h).

    with Server([op_a, op_b], gamma_inv=[g_a, None], pool_bytes=8 << 30, max_batch=64) as srv:
        t = srv.submit(0, m, y)        # m, y: [nvec][N_t][N_m] float32, host (pinned) or CUDA
        srv.wait(t)
        print(srv.stats())

The scheduler admits requests in arrival order under the device-memory
pool, batches each operator's admitted requests whenever that operator's
previous batch has finished (continuous batching), and runs the operators'
batches concurrently on their own streams.  Tensors passed to submit must
stay alive until their request completes; this wrapper keeps references.
"""
import ctypes

from . import _lib
from .operator import _ptr_and_stream

STATES = {0: "waiting", 1: "admitted", 2: "running", 3: "done", 4: "failed"}
FAULT_BATCH, FAULT_ADMIT = 1, 2


class Server:
    def __init__(self, operators, gamma_inv=None, pool_bytes=1 << 30, max_batch=64):
        self._lib = _lib.load()
        self.operators = list(operators)
        n = len(self.operators)
        ops = (ctypes.c_void_p * n)(*[o.handle.value for o in self.operators])
        self._keep = {}
        gam = None
        if gamma_inv is not None:
            ptrs = []
            for o, g in zip(self.operators, gamma_inv):
                if g is None:
                    ptrs.append(None)
                else:
                    if not (hasattr(g, "is_cuda") and g.is_cuda):
                        raise ValueError("gamma_inv must be CUDA tensors (or None)")
                    if tuple(g.shape) != (o.N_t, o.N_d):
                        raise ValueError("gamma_inv has shape %s" % (tuple(g.shape),))
                    ptrs.append(g.data_ptr())
            self._gamma = list(gamma_inv)
            gam = (ctypes.c_void_p * n)(*ptrs)
        h = ctypes.c_void_p()
        _lib.check(self._lib.btt_server_create(ctypes.byref(h), ops, gam, n, int(pool_bytes), int(max_batch)))
        self._h = h
        self.max_batch = int(max_batch)

    def submit(self, op, m, y):
        """Queue y = H_op m; returns a ticket.  m, y: [nvec][N_t][N_m] float32."""
        o = self.operators[op]
        if m.ndim != 3 or tuple(m.shape[1:]) != (o.N_t, o.N_m) or tuple(y.shape) != tuple(m.shape):
            raise ValueError("m and y must have shape [nvec][%d][%d]" % (o.N_t, o.N_m))
        if str(m.dtype).replace("torch.", "") != "float32" or str(y.dtype).replace("torch.", "") != "float32":
            raise TypeError("vectors must be float32")
        pm, _ = _ptr_and_stream(m, 0)
        py, _ = _ptr_and_stream(y, 0)
        t = ctypes.c_longlong()
        _lib.check(self._lib.btt_server_submit(self._h, int(op), pm, py, int(m.shape[0]), ctypes.byref(t)))
        self._keep[t.value] = (m, y)
        return t.value

    def wait(self, ticket, timeout=-1.0):
        """Blocks until the request is done; raises BttError if it failed or timed out."""
        st = self._lib.btt_server_wait(self._h, ticket, float(timeout))
        if st != _lib.BTT_ERR_TIMEOUT:
            self._keep.pop(ticket, None)
        _lib.check(st)

    def poll(self, ticket):
        s = ctypes.c_int()
        _lib.check(self._lib.btt_server_poll(self._h, ticket, ctypes.byref(s)))
        return STATES[s.value]

    def stats(self, reset=False):
        st = _lib.ServingStats()
        _lib.check(self._lib.btt_server_stats(self._h, ctypes.byref(st), 1 if reset else 0))
        return st.as_dict()

    def inject(self, fault):
        """Host-side fault injection: FAULT_BATCH or FAULT_ADMIT for the next one."""
        _lib.check(self._lib.btt_server_inject(self._h, int(fault)))

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.btt_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
