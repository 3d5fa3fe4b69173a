"""FP64 CPU oracle for the accelerated Jacobi method (arXiv 2407.03272).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the product path never does.  It
shares no code with the CUDA library (``paper_2407_03272_gb300``) and neither
imports the other.

``solve`` runs Algorithm alg-jacobi (Section 3) with the adaptive restart of
Algorithm alg-apg-re (Section 2.2) in plain C, FP64, one thread, with a
diagonal J (eq. J-diag and its variants) or a block-diagonal J
(eq. J-blkdiag, built by ``j_blkdiag``).  Dense helpers
for tiny inputs (the step constant L = lambda_max(D^-1/2 Q D^-1/2), f(x))
live in ``oracle.dense``; ``oracle.schedule`` checks a restart schedule
against the rule of Algorithm alg-apg-re.
"""
import ctypes
import numpy as np

from . import build as _build

STOP_NONE, STOP_RELRES, STOP_OBJGAP = 0, 1, 2

_libs = {}


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("b", ctypes.c_void_p), ("J", ctypes.c_void_p),
                ("x0", ctypes.c_void_p), ("is_restart", ctypes.c_int), ("momentum", ctypes.c_int),
                ("K0", ctypes.c_int64), ("maxit", ctypes.c_int64), ("stop", ctypes.c_int),
                ("tol", ctypes.c_double), ("fstar", ctypes.c_double), ("forced", ctypes.c_void_p),
                ("bs", ctypes.c_int64), ("Jblk", ctypes.c_void_p)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("restarts", ctypes.c_int64), ("relres", ctypes.c_double),
                ("f", ctypes.c_double), ("converged", ctypes.c_int)]


class _Trace(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("alpha", "beta", "d", "restart", "f", "relres", "gnorm", "x", "y", "dxnorm", "gfloor")]


def host_cores():
    """Cores this process may run on (its CPU affinity)."""
    import os
    return len(os.sched_getaffinity(0))


def lib(omp=False):
    """The correctness build, or (omp=True) the OpenMP timing build of the
    same source, which computes the same bits on all the host's cores."""
    if omp not in _libs:
        path = _build.build_omp() if omp else _build.build()
        L = ctypes.CDLL(path)
        L.orc_spmv.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5
        L.orc_j_absrowsum.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 4
        L.orc_j_scaled_diag.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_void_p]
        L.orc_aj_solve.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.POINTER(_Info),
                                   ctypes.POINTER(_Trace)]
        L.orc_aj_solve.restype = ctypes.c_int
        L.orc_pcg_solve.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int64, ctypes.c_double,
                                                                              ctypes.c_void_p, ctypes.c_void_p,
                                                                              ctypes.c_void_p]
        L.orc_pcg_solve.restype = ctypes.c_int
        _libs[omp] = L
    return _libs[omp]


def _p(a):
    return None if a is None else a.ctypes.data


def _csr(Q):
    rp = np.ascontiguousarray(Q["row_ptr"], dtype=np.int32)
    ci = np.ascontiguousarray(Q["col"], dtype=np.int32)
    v = np.ascontiguousarray(Q["val"], dtype=np.float64)
    return int(Q["n"]), rp, ci, v


def spmv(Q, y):
    """Q @ y, each row summed in ascending column order."""
    n, rp, ci, v = _csr(Q)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.empty(n, dtype=np.float64)
    lib().orc_spmv(n, _p(rp), _p(ci), _p(v), _p(y), _p(out))
    return out


def j_absrowsum(Q):
    """eq. J-diag: J_kk = Q_kk + sum_{j != k} |Q_kj| (zero row -> 1)."""
    n, rp, ci, v = _csr(Q)
    J = np.empty(n, dtype=np.float64)
    lib().orc_j_absrowsum(n, _p(rp), _p(ci), _p(v), _p(J))
    return J


def j_scaled_diag(Q, c):
    """J_kk = c * Q_kk (zero diagonal -> 1).  c = L for the L*D proximal term,
    c = 1/omega for weighted Jacobi (eq. weighted-jacobi)."""
    n, rp, ci, v = _csr(Q)
    J = np.empty(n, dtype=np.float64)
    lib().orc_j_scaled_diag(n, _p(rp), _p(ci), _p(v), float(c), _p(J))
    return J


def j_blkdiag(Q, bs):
    """eq. J-blkdiag with s = ceil(n / bs) blocks of bs consecutive rows:
    J^{ii} = Q^{ii} + (sum_{j != i} ||Q^{ij}||_2) I, the spectral norm of each
    off-diagonal block by a dense SVD (numpy.linalg.norm(., 2)).

    Reading where the paper is silent: a block whose J^{ii} is singular (a
    part of Q wholly inside the block that is itself singular, e.g. a
    component of a graph Laplacian, or a zero row) gets eq. J-diag's diagonal
    instead; singular means lambda_min(J^{ii}) <= 1e-12 * max_k J^{ii}_kk.

    Returns an (s, bs, bs) array; the last block's rows and columns beyond n
    hold the identity."""
    n, rp, ci, v = _csr(Q)
    bs = int(bs)
    s = (n + bs - 1) // bs
    out = np.zeros((s, bs, bs))
    jd = j_absrowsum(Q)
    for ib in range(s):
        r0 = ib * bs
        nb = min(bs, n - r0)
        D = np.zeros((bs, bs))
        off = {}
        for k in range(nb):
            i = r0 + k
            for p in range(rp[i], rp[i + 1]):
                c = int(ci[p])
                jb = c // bs
                if jb == ib:
                    D[k, c - r0] += v[p]
                else:
                    A = off.setdefault(jb, np.zeros((bs, bs)))
                    A[k, c - jb * bs] += v[p]
        c_i = sum(np.linalg.norm(off[jb], 2) for jb in sorted(off))
        Jb = D[:nb, :nb] + c_i * np.eye(nb)
        if nb > 0 and np.linalg.eigvalsh(Jb)[0] <= 1e-12 * max(np.max(np.diag(Jb)), 0.0):
            Jb = np.diag(jd[r0:r0 + nb])
        out[ib, :nb, :nb] = Jb
        for k in range(nb, bs):
            out[ib, k, k] = 1.0
    return out


def pcg(Q, b, *, maxit=1000, tol=1e-8, x0=None):
    """The comparator of Section 4.2: conjugate gradients preconditioned by
    M = diag(Q) (Saad's Alg. 9.1), stopping when the recursive residual
    satisfies ||r^t|| <= tol ||b|| or after maxit iterations.  Returns a dict
    with x, iters and rr (||r^t|| for t = 0 .. iters)."""
    n, rp, ci, v = _csr(Q)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    x = np.empty(n, dtype=np.float64)
    rr = np.full(maxit + 1, np.nan)
    it = ctypes.c_int64()
    rc = lib().orc_pcg_solve(n, _p(rp), _p(ci), _p(v), _p(b), _p(x0a), int(maxit), float(tol), _p(x),
                             ctypes.byref(it), _p(rr))
    if rc != 0:
        raise ValueError("oracle rejected the input")
    return dict(x=x, iters=it.value, rr=rr[: it.value + 1])


def solve(Q, b, J=None, *, Jblk=None, restart=True, momentum=True, K0=2, maxit=1000, stop=STOP_RELRES,
          tol=1e-8, fstar=0.0, x0=None, forced=None, trace=False, trace_iterates=False, omp=False):
    """Run Algorithm alg-jacobi with the diagonal J or, if given, the block
    diagonal Jblk (from ``j_blkdiag``); returns a dict with x, iters,
    restarts, relres, f, converged and (trace=True) per-iteration arrays
    indexed by t.  omp=True runs the OpenMP timing build (same bits)."""
    n, rp, ci, v = _csr(Q)
    b = np.ascontiguousarray(b, dtype=np.float64)
    bs = 0
    if Jblk is not None:
        Jblk = np.ascontiguousarray(Jblk, dtype=np.float64)
        bs = int(Jblk.shape[1])
        J = np.ones(max(n, 1))
    J = np.ascontiguousarray(J, dtype=np.float64)
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    fa = None
    if forced is not None:
        fa = np.zeros(maxit + 1, dtype=np.uint8)
        for t in forced:
            if 1 <= t <= maxit:
                fa[t] = 1
    P = _Params(n, _p(rp), _p(ci), _p(v), _p(b), _p(J), _p(x0a), int(bool(restart)),
                int(bool(momentum)), int(K0), int(maxit), int(stop), float(tol), float(fstar), _p(fa),
                bs, _p(Jblk))
    info = _Info()
    x = np.empty(n, dtype=np.float64)
    tr = {}
    T = None
    if trace or trace_iterates:
        m = maxit + 1
        for k in ("alpha", "beta", "d", "f", "relres", "gnorm", "dxnorm", "gfloor"):
            tr[k] = np.full(m, np.nan)
        tr["restart"] = np.zeros(m, dtype=np.uint8)
        if trace_iterates:
            tr["x"] = np.full((m, n), np.nan)
            tr["y"] = np.full((m, n), np.nan)
        T = _Trace(*[_p(tr.get(k)) for k in ("alpha", "beta", "d", "restart", "f", "relres",
                                              "gnorm", "x", "y", "dxnorm", "gfloor")])
    rc = lib(omp).orc_aj_solve(ctypes.byref(P), _p(x), ctypes.byref(info),
                               ctypes.byref(T) if T is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the input")
    out = dict(x=x, iters=info.iters, restarts=info.restarts, relres=info.relres, f=info.f,
               converged=bool(info.converged))
    if tr:
        t = info.iters
        out["trace"] = {k: (a[: t + 1] if a.ndim == 1 else a[: t + 1]) for k, a in tr.items()}
    return out
