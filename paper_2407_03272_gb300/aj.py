"""ctypes binding of libaj (include/aj.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); pointers
and sizes are passed through unchanged.  If the library is missing or fails
to load, every call raises -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

AJ_OK, AJ_EINVAL, AJ_ENOMEM, AJ_ECUDA = 0, -1, -2, -3
AJ_EMAXIT, AJ_EDIVERGED, AJ_ENONFINITE, AJ_ETIMEOUT, AJ_EBUSY = -4, -5, -6, -7, -8
AJ_PENDING = 1
AJ_J_ABSROWSUM, AJ_J_SCALED_DIAG, AJ_J_BLKDIAG = 0, 1, 2
AJ_RESTART_NONE, AJ_RESTART_ADAPTIVE = 0, 1
AJ_STOP_RELRES, AJ_STOP_OBJGAP, AJ_STOP_NONE = 0, 1, 2
AJ_FP64, AJ_DF64, AJ_FP32_IR, AJ_BF16_IR = 0, 1, 2, 3
AJ_FMT_AUTO, AJ_FMT_CSR, AJ_FMT_SELL, AJ_FMT_STENCIL = 0, 1, 2, 3
AJ_SWEEP_AUTO, AJ_SWEEP_LAZY, AJ_SWEEP_STORED, AJ_SWEEP_DELTA, AJ_SWEEP_Y = 0, 1, 2, 3, 4
AJ_REORDER_AUTO, AJ_REORDER_NONE, AJ_REORDER_RCM = 0, 1, 2
AJ_NOALLOC_MAX_N = 131072

PRECISIONS = {"fp64": AJ_FP64, "df64": AJ_DF64, "fp32_ir": AJ_FP32_IR, "bf16_ir": AJ_BF16_IR}


class aj_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class aj_params(ctypes.Structure):
    _fields_ = [("j_policy", ctypes.c_int), ("L", ctypes.c_double), ("L_margin", ctypes.c_double),
                ("restart", ctypes.c_int), ("momentum", ctypes.c_int), ("K0", ctypes.c_int64),
                ("tol", ctypes.c_double), ("stop", ctypes.c_int), ("fstar", ctypes.c_double),
                ("maxit", ctypes.c_int64), ("precision", ctypes.c_int), ("format", ctypes.c_int),
                ("x0", ctypes.c_void_p), ("x0_on_device", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int64),
                ("grid_ctas", ctypes.c_int), ("sweep_form", ctypes.c_int),
                ("sell_sigma", ctypes.c_int), ("sell_lmax", ctypes.c_int), ("reorder", ctypes.c_int),
                ("j_block", ctypes.c_int), ("sell_c", ctypes.c_int)]


class aj_tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("format", "sell_c", "sell_sigma", "sell_lmax", "lanes_per_row",
                                            "rows_per_cta", "threads_per_cta", "ctas_per_sm", "grid",
                                            "sweep_form", "tuned", "pad_")] + [("fill_ratio", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class aj_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("restarts", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("outer", ctypes.c_int64), ("relres", ctypes.c_double), ("objgap", ctypes.c_double),
                ("L_used", ctypes.c_double), ("ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class aj_server_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("peak_active", ctypes.c_int64), ("peak_bytes", ctypes.c_uint64),
                ("in_use_bytes", ctypes.c_uint64), ("queued", ctypes.c_int64), ("kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AJError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = lib().aj_strerror(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s (%d)" % (what, msg, status))


_lib = None
LIB_PATH = None

# (name, restype, argtypes) of every entry point declared in include/aj.h
SIGNATURES = [
    ("aj_params_default", None, [ctypes.POINTER(aj_params)]),
    ("aj_create", ctypes.c_int, [ctypes.POINTER(aj_csr), ctypes.c_void_p, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_void_p)]),
    ("aj_set", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(aj_params)]),
    ("aj_get_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(aj_tuning)]),
    ("aj_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("aj_get_order", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]),
    ("aj_get_format", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    ("aj_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(aj_info)]),
    ("aj_solve_rhs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(aj_info)]),
    ("aj_solve_batch", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                      ctypes.POINTER(aj_info)]),
    ("aj_server_create", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("aj_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    ("aj_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(aj_info)]),
    ("aj_submit_csr", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(aj_csr), ctypes.c_void_p, ctypes.c_int,
                                     ctypes.POINTER(aj_params), ctypes.POINTER(ctypes.c_uint64)]),
    ("aj_server_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double]),
    ("aj_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(aj_server_stats)]),
    ("aj_server_destroy", None, [ctypes.c_void_p]),
    ("aj_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("aj_set_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("aj_restart_log", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    ("aj_pcg_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(aj_info)]),
    ("aj_destroy", None, [ctypes.c_void_p]),
    ("aj_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("aj_kernel_launches", ctypes.c_uint64, []),
    ("aj_cache_stats", None, [ctypes.POINTER(ctypes.c_uint64)] * 4),
    ("aj_solve_noalloc", ctypes.c_int, [ctypes.POINTER(aj_csr), ctypes.c_void_p, ctypes.POINTER(aj_params),
                                        ctypes.c_void_p, ctypes.POINTER(aj_info), ctypes.c_void_p]),
    ("aj_test_barrier_stall", ctypes.c_int, [ctypes.c_int, ctypes.c_double]),
    ("aj_test_alloc_fail", ctypes.c_int, [ctypes.c_int64]),
]


def lib(path=None):
    """Load libaj (building it first if needed).  Raises if that fails."""
    global _lib, LIB_PATH
    if _lib is None:
        p = path or os.environ.get("AJ_LIB") or _build.build()
        L = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        LIB_PATH = p
    return _lib


def _check(st, what):
    if st != AJ_OK:
        raise AJError(st, what)


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError("expected a numpy array or a torch tensor")


def params(**kw):
    p = aj_params()
    lib().aj_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "x0":
            continue
        setattr(p, k, v)
    return p


class Context:
    """One linear system Q x = b (1..4 right-hand sides) living on the GPU."""

    def __init__(self, row_ptr, col, val, b, n=None, nrhs=1, stream=None):
        L = lib()
        rp, d0 = _ptr(row_ptr)
        ci, d1 = _ptr(col)
        v, d2 = _ptr(val)
        bp, d3 = _ptr(b)
        if len({d0, d1, d2, d3}) != 1:
            raise ValueError("Q and b must all be on the host or all on the device")
        n = int(len(row_ptr) - 1) if n is None else int(n)
        nnz = int(len(col))
        self.n, self.nnz, self.nrhs = n, nnz, int(nrhs)
        self._keep = (row_ptr, col, val, b)
        csr = aj_csr(n, nnz, rp, ci, v, d0)
        h = ctypes.c_void_p()
        _check(L.aj_create(ctypes.byref(csr), bp, self.nrhs, ctypes.byref(h)), "aj_create")
        self._h = h
        self._keep = None
        self._x0 = None
        if stream is not None:
            self.set_stream(stream)

    @property
    def handle(self):
        return self._h

    def set(self, x0=None, **kw):
        p = params(**kw)
        if x0 is not None:
            xp, dev = _ptr(x0)
            p.x0, p.x0_on_device = xp, dev
            self._x0 = x0
        _check(lib().aj_set(self._h, ctypes.byref(p)), "aj_set")
        return self

    def format(self):
        """(format, sigma, lmax, fill_ratio) chosen by aj_set."""
        f, sg, lm, fr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().aj_get_format(self._h, ctypes.byref(f), ctypes.byref(sg), ctypes.byref(lm),
                                   ctypes.byref(fr)), "aj_get_format")
        return f.value, sg.value, lm.value, fr.value

    def tuning(self):
        """The fused sweep's configuration aj_set chose (aj_get_tuning), as a dict."""
        t = aj_tuning()
        _check(lib().aj_get_tuning(self._h, ctypes.byref(t)), "aj_get_tuning")
        return t.as_dict()

    def order(self):
        """(reordered, span_before, span_after) decided by aj_set."""
        o, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(lib().aj_get_order(self._h, ctypes.byref(o), ctypes.byref(a), ctypes.byref(b)), "aj_get_order")
        return o.value, a.value, b.value

    def set_stream(self, stream):
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        _check(lib().aj_set_stream(self._h, ctypes.c_void_p(s)), "aj_set_stream")

    def solve(self, out=None, per_rhs=False, raise_on_error=False):
        """Returns (x, info).  out: preallocated float64 array/tensor of n*nrhs
        (column-major); default a new numpy array on the host."""
        if out is None:
            out = np.empty(self.n * self.nrhs if self.nrhs > 1 else self.n, dtype=np.float64)
        xp, dev = _ptr(out)
        if per_rhs:
            infos = (aj_info * self.nrhs)()
            st = lib().aj_solve_rhs(self._h, xp, dev, infos)
            info = [i.as_dict() for i in infos]
        else:
            inf = aj_info()
            st = lib().aj_solve(self._h, xp, dev, ctypes.byref(inf))
            info = inf.as_dict()
        if st not in (AJ_OK, AJ_EMAXIT, AJ_EDIVERGED, AJ_ENONFINITE) or (raise_on_error and st != AJ_OK):
            raise AJError(st, "aj_solve")
        return out, info

    def pcg_solve(self, out=None):
        """Sec. 4.2's comparator, diagonally preconditioned CG on the same
        system (aj_pcg_solve); returns (x, info)."""
        if out is None:
            out = np.empty(self.n, dtype=np.float64)
        xp, dev = _ptr(out)
        inf = aj_info()
        st = lib().aj_pcg_solve(self._h, xp, dev, ctypes.byref(inf))
        if st not in (AJ_OK, AJ_EMAXIT, AJ_ENONFINITE):
            raise AJError(st, "aj_pcg_solve")
        return out, inf.as_dict()

    def restart_log(self, rhs=0):
        cnt = ctypes.c_int64()
        _check(lib().aj_restart_log(self._h, rhs, None, 0, ctypes.byref(cnt)), "aj_restart_log")
        buf = (ctypes.c_int64 * max(1, cnt.value))()
        _check(lib().aj_restart_log(self._h, rhs, buf, cnt.value, ctypes.byref(cnt)), "aj_restart_log")
        return [int(buf[i]) for i in range(cnt.value)]

    def get_state(self):
        size = ctypes.c_size_t()
        _check(lib().aj_get_state(self._h, None, ctypes.byref(size)), "aj_get_state")
        buf = ctypes.create_string_buffer(size.value)
        _check(lib().aj_get_state(self._h, buf, ctypes.byref(size)), "aj_get_state")
        return buf.raw

    def set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().aj_set_state(self._h, buf, len(blob)), "aj_set_state")

    def close(self):
        if getattr(self, "_h", None):
            lib().aj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_csr(Q, b, nrhs=1, device=None):
    """Context from a synth-style CSR dict and b (numpy).  device='cuda' first
    copies the arrays to the GPU with torch (memory plumbing only)."""
    rp = np.ascontiguousarray(Q["row_ptr"], np.int32)
    ci = np.ascontiguousarray(Q["col"], np.int32)
    v = np.ascontiguousarray(Q["val"], np.float64)
    bb = np.ascontiguousarray(b, np.float64)
    if device is not None:
        import torch
        t = [torch.from_numpy(a).to(device) for a in (rp, ci, v, bb)]
        return Context(*t, n=Q["n"], nrhs=nrhs)
    return Context(rp, ci, v, bb, n=Q["n"], nrhs=nrhs)


def solve_batch(ctxs, outs, on_device=False):
    n = len(ctxs)
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    ps = (ctypes.c_void_p * n)(*[_ptr(o)[0] for o in outs])
    infos = (aj_info * n)()
    st = lib().aj_solve_batch(hs, n, ps, int(on_device), infos)
    if st not in (AJ_OK, AJ_EMAXIT, AJ_EDIVERGED, AJ_ENONFINITE):
        raise AJError(st, "aj_solve_batch")
    return [i.as_dict() for i in infos]


def _check_noalloc_args(row_ptr, col, val, b, x_out, x0):
    """The kernels of aj_solve_noalloc read row_ptr (n + 1 int32), col (nnz
    int32), val (nnz float64), b and x0 (n float64) and write x_out (n
    float64) through raw pointers: refuse anything else before the call."""
    import torch
    named = [("row_ptr", row_ptr, torch.int32), ("col", col, torch.int32), ("val", val, torch.float64),
             ("b", b, torch.float64), ("x_out", x_out, torch.float64)]
    if x0 is not None:
        named.append(("x0", x0, torch.float64))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError("aj_solve_noalloc: %s must be a torch tensor" % name)
        if t.dtype != dt:
            raise ValueError("aj_solve_noalloc: %s must be %s, not %s" % (name, dt, t.dtype))
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError("aj_solve_noalloc: %s must be a contiguous vector" % name)
    n = row_ptr.numel() - 1
    if n < 0:
        raise ValueError("aj_solve_noalloc: row_ptr needs n + 1 entries")
    if val.numel() != col.numel():
        raise ValueError("aj_solve_noalloc: val and col differ in length")
    for name, t, _ in named[3:]:
        if t.numel() < n:
            raise ValueError("aj_solve_noalloc: %s holds %d entries, n = %d" % (name, t.numel(), n))
    dev = None
    for name, t, _ in named:
        if not t.is_cuda:
            raise ValueError("aj_solve_noalloc takes device arrays only (%s is on %s)" % (name, t.device))
        dev = t.device if dev is None else dev
        if t.device != dev:
            raise ValueError("aj_solve_noalloc: %s is on %s, row_ptr on %s" % (name, t.device, dev))
    if dev.index != torch.cuda.current_device():
        raise ValueError("aj_solve_noalloc: the arrays are on %s, the current device is cuda:%d"
                         % (dev, torch.cuda.current_device()))


def solve_noalloc(row_ptr, col, val, b, x_out, stream=None, **kw):
    """aj_solve_noalloc on device tensors: the FP64 solve for one right-hand
    side with the library's fixed scratch array (no device allocation inside
    the call).  Returns (status, info dict).  The tensors' types, lengths and
    device are checked first (ValueError)."""
    x0 = kw.get("x0")
    _check_noalloc_args(row_ptr, col, val, b, x_out, x0)
    ptrs = [_ptr(a) for a in (row_ptr, col, val, b, x_out)]
    p = params(**kw)
    if x0 is not None:
        p.x0, p.x0_on_device = _ptr(x0)
    csr = aj_csr(int(len(row_ptr) - 1), int(len(col)), ptrs[0][0], ptrs[1][0], ptrs[2][0], 1)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    inf = aj_info()
    st = lib().aj_solve_noalloc(ctypes.byref(csr), ptrs[3][0], ctypes.byref(p), ptrs[4][0],
                                ctypes.byref(inf), ctypes.c_void_p(s))
    return st, inf.as_dict()


def cache_stats():
    """Hits and misses of aj_set's ordering and autotuner caches (aj_cache_stats)."""
    v = [ctypes.c_uint64() for _ in range(4)]
    lib().aj_cache_stats(*[ctypes.byref(x) for x in v])
    return dict(zip(("order_hits", "order_misses", "tune_hits", "tune_misses"), (x.value for x in v)))


def inject_barrier_stall(cta, timeout_ms):
    """Failure-detection hook (aj_test_barrier_stall): CTA `cta` of the next
    persistent solve withholds its first barrier arrival, and that launch's
    barrier waits give up after timeout_ms."""
    _check(lib().aj_test_barrier_stall(int(cta), float(timeout_ms)), "aj_test_barrier_stall")


def inject_alloc_failure(after):
    """Failure-detection hook (aj_test_alloc_fail): the device allocation
    after `after` more successful ones fails once (-1 disarms)."""
    _check(lib().aj_test_alloc_fail(int(after)), "aj_test_alloc_fail")


class Server:
    """Continuous-batching solve server (aj_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots):
        h = ctypes.c_void_p()
        _check(lib().aj_server_create(ctypes.c_size_t(int(hbm_budget_bytes)), int(max_slots),
                                      ctypes.byref(h)), "aj_server_create")
        self._h = h
        self._meta = {}

    def submit(self, ctx):
        t = ctypes.c_uint64()
        _check(lib().aj_submit(self._h, ctx.handle, ctypes.byref(t)), "aj_submit")
        self._meta[t.value] = (ctx.n, ctx.nrhs, ctx)
        return t.value

    def submit_csr(self, Q, b, nrhs=1, **kw):
        """Q: synth-style CSR dict (host numpy); b: n*nrhs column-major."""
        rp = np.ascontiguousarray(Q["row_ptr"], np.int32)
        ci = np.ascontiguousarray(Q["col"], np.int32)
        v = np.ascontiguousarray(Q["val"], np.float64)
        bb = np.ascontiguousarray(b, np.float64)
        csr = aj_csr(int(Q["n"]), int(ci.size), rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 0)
        p = params(**kw)
        x0 = kw.get("x0")
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, np.float64)
            p.x0, p.x0_on_device = x0.ctypes.data, 0
        t = ctypes.c_uint64()
        _check(lib().aj_submit_csr(self._h, ctypes.byref(csr), bb.ctypes.data, int(nrhs), ctypes.byref(p),
                                   ctypes.byref(t)), "aj_submit_csr")
        self._meta[t.value] = (int(Q["n"]), int(nrhs), None)
        return t.value

    def poll(self, ticket):
        """None while pending, else (status, x, info)."""
        n, nrhs, _ = self._meta[ticket]
        x = np.empty(n * nrhs, dtype=np.float64)
        inf = aj_info()
        st = lib().aj_poll(self._h, ctypes.c_uint64(ticket), x.ctypes.data, ctypes.byref(inf))
        if st == AJ_PENDING:
            return None
        if st == AJ_EINVAL:
            raise AJError(st, "aj_poll")
        del self._meta[ticket]
        return st, x, inf.as_dict()

    def wait(self, ticket, timeout_ms=-1.0):
        return lib().aj_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout_ms))

    def result(self, ticket):
        """Block until the request finishes; (status, x, info)."""
        st = self.wait(ticket)
        if st not in (AJ_OK, AJ_PENDING):
            raise AJError(st, "aj_server_wait")
        return self.poll(ticket)

    def stats(self):
        st = aj_server_stats()
        _check(lib().aj_server_get_stats(self._h, ctypes.byref(st)), "aj_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().aj_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
