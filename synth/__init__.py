"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds matrices and vectors only.  It holds none of the
accelerated-Jacobi arithmetic, and both the FP64 oracle and the CUDA library
take its outputs as plain inputs.  Random numbers come from numpy's PCG64 bit
generator with an explicit seed.

A CSR matrix is a dict ``{"n", "row_ptr" (int32, n+1), "col" (int32, nnz),
"val" (float64, nnz)}``.  Column indices ascend within every row.

Workloads (the paper's data sets are not in this container, so these stand in
for them):
  * ``poisson2d(N)``: 5-point Dirichlet Laplacian on an N x N grid (diagonal 4,
    neighbours -1, natural row-major ordering).  Its eigenvalues are known in
    closed form.
  * ``poisson3d(N)``: the 7-point analogue (diagonal 6).
  * ``sdd(n)``: the strictly diagonally dominant matrix of Section 4.1.  It has
    n on the diagonal and -1 elsewhere, and with b = 1 the exact solution is 1.
  * ``chung_lu_laplacian``: the weighted Laplacian D - W of a Chung-Lu
    power-law graph.  It stands in for the SuiteSparse graphs of Section 4.2.
    Isolated vertices are kept as empty rows.
  * ``rgg_knn_laplacian``: the Laplacian of a symmetrised k-nearest-neighbour
    random geometric graph in the unit square, with Gaussian weights.
"""
import numpy as np

try:  # the rhs b = Q x* uses a library sparse product; it is input construction only
    import scipy.sparse as _sp
except Exception:  # pragma: no cover
    _sp = None


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def poisson2d(N):
    """5-point Dirichlet Laplacian on an N x N grid, row r = j*N + i."""
    n = N * N
    r = np.arange(n, dtype=np.int64)
    i = r % N
    j = r // N
    offs = [(-N, j > 0), (-1, i > 0), (0, np.ones(n, bool)), (1, i < N - 1), (N, j < N - 1)]
    return _stencil(n, r, offs, 4.0)


def poisson3d(N):
    """7-point Dirichlet Laplacian on an N^3 grid, row r = (k*N + j)*N + i."""
    n = N * N * N
    r = np.arange(n, dtype=np.int64)
    i = r % N
    j = (r // N) % N
    k = r // (N * N)
    NN = N * N
    offs = [(-NN, k > 0), (-N, j > 0), (-1, i > 0), (0, np.ones(n, bool)),
            (1, i < N - 1), (N, j < N - 1), (NN, k < N - 1)]
    return _stencil(n, r, offs, 6.0)


def _stencil(n, r, offs, diag):
    m = len(offs)
    mask = np.empty((n, m), dtype=bool)
    for c, (o, ok) in enumerate(offs):
        mask[:, c] = ok
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    cols = np.empty((n, m), dtype=np.int32)
    vals = np.empty((n, m), dtype=np.float64)
    for c, (o, ok) in enumerate(offs):
        cols[:, c] = (r + o).astype(np.int32) if o != 0 else r.astype(np.int32)
        vals[:, c] = diag if o == 0 else -1.0
    col = cols[mask]
    val = vals[mask]
    assert col.size == nnz
    return {"n": n, "row_ptr": row_ptr.astype(np.int32), "col": col, "val": val}


def sdd(n):
    """Q = (n + 1) I - 1 1^T: n on the diagonal, -1 off it (Section 4.1)."""
    row_ptr = (np.arange(n + 1, dtype=np.int64) * n).astype(np.int32)
    col = np.tile(np.arange(n, dtype=np.int32), n)
    val = np.full(n * n, -1.0)
    val[np.arange(n) * n + np.arange(n)] = float(n)
    return {"n": n, "row_ptr": row_ptr, "col": col, "val": val}


def from_edges(n, u, v, w):
    """Laplacian D - W of an undirected weighted graph with edge list (u, v, w),
    u != v and no duplicate pairs.  Isolated vertices get empty rows."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    w = np.asarray(w, np.float64)
    # weighted degrees, summed in edge order (all u-ends, then all v-ends)
    deg = np.bincount(np.concatenate([u, v]), weights=np.concatenate([w, w]), minlength=n)
    dr = np.nonzero(deg != 0)[0]
    rows = np.concatenate([u, v, dr])
    cols = np.concatenate([v, u, dr])
    vals = np.concatenate([-w, -w, deg[dr]])
    if rows.size >= 2 ** 31:
        raise ValueError("nnz exceeds int32 indices")
    # COO -> CSR with ascending columns (no duplicate pairs, so nothing is summed)
    A = _sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    return {"n": n, "row_ptr": A.indptr.astype(np.int32), "col": A.indices.astype(np.int32),
            "val": np.asarray(A.data, np.float64)}


def with_hubs(Q, hubs, degree, seed=7, wlo=0.5, whi=1.5):
    """The Laplacian of Q's graph with each vertex in ``hubs`` joined to
    ``degree`` more distinct vertices, drawn uniformly among those it is not yet
    joined to, with U(wlo, whi) weights (a planted hub: rows of ``degree`` and
    more entries).  Q must be a graph Laplacian (from ``from_edges``)."""
    rng = _rng(seed)
    n = int(Q["n"])
    rp, ci, v = Q["row_ptr"], Q["col"], Q["val"]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    keep = rows < ci  # each edge once, from its lower end
    u, w_, wt = rows[keep], ci[keep].astype(np.int64), -v[keep]
    have = set(zip(u.tolist(), w_.tolist()))
    eu, ev, ew = [u], [w_], [wt]
    for h in hubs:
        h = int(h)
        cand = rng.permutation(n)
        picked = []
        for c in cand.tolist():
            if c == h or (min(c, h), max(c, h)) in have:
                continue
            picked.append(c)
            have.add((min(c, h), max(c, h)))
            if len(picked) == degree:
                break
        p = np.asarray(picked, np.int64)
        eu.append(np.minimum(p, h))
        ev.append(np.maximum(p, h))
        ew.append(rng.uniform(wlo, whi, p.size))
    return from_edges(n, np.concatenate(eu), np.concatenate(ev), np.concatenate(ew))


def _inverse_cdf(cdf, u):
    """searchsorted(cdf, u, side="right"), with the queries sorted first so
    that the binary searches walk the table in order (same result)."""
    order = np.argsort(u)
    out = np.empty(u.size, dtype=np.int64)
    out[order] = np.searchsorted(cdf, u[order], side="right")
    return out


def chung_lu_laplacian(n, mean_degree=16.0, exponent=2.5, seed=3, wlo=0.5, whi=1.5):
    """Weighted Laplacian of a Chung-Lu graph.

    Expected degrees are w_i proportional to (i + i0)^(-1/(exponent-1)), with
    mean ``mean_degree``.  The offset i0 is chosen so that w_max = sqrt(sum w).
    Endpoint pairs are drawn independently in proportion to w.  Self-loops are
    dropped, and of each duplicate pair the first drawn is kept with its
    U(wlo, whi) weight.  The sample count is rescaled until the mean degree is
    within 1 % of ``mean_degree``.
    """
    rng = _rng(seed)
    gamma = 1.0 / (exponent - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def shape(i0):
        s = (idx + i0) ** (-gamma)
        return s * (mean_degree * n / s.sum())

    lo, hi = 0.0, float(n)
    for _ in range(60):  # bisection on i0 so that w_0 = sqrt(sum w)
        mid = 0.5 * (lo + hi)
        w = shape(max(mid, 1e-9))
        if w[0] > np.sqrt(w.sum()):
            lo = mid
        else:
            hi = mid
    w = shape(max(hi, 1e-9))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    target = mean_degree * n / 2.0
    m = int(round(target))
    for _ in range(6):
        a = _inverse_cdf(cdf, rng.random(m))
        b = _inverse_cdf(cdf, rng.random(m))
        np.minimum(a, n - 1, out=a)
        np.minimum(b, n - 1, out=b)
        wt = rng.uniform(wlo, whi, m)
        keep = a != b
        a, b, wt = a[keep], b[keep], wt[keep]
        key = np.minimum(a, b).astype(np.int64) * n + np.maximum(a, b)
        _, first = np.unique(key, return_index=True)
        ne = first.size
        if abs(ne - target) <= 0.01 * target:
            break
        m = int(round(m * target / ne))
    first.sort()
    u = np.minimum(a, b)[first]
    v = np.maximum(a, b)[first]
    return from_edges(n, u, v, wt[first])


def rgg_knn_laplacian(n, k=8, seed=4):
    """Laplacian of a random geometric graph: n points U[0,1]^2, each joined to
    its k nearest neighbours (union symmetrisation), weight exp(-d^2/sigma^2)
    with sigma the median k-th neighbour distance."""
    from scipy.spatial import cKDTree
    rng = _rng(seed)
    P = rng.random((n, 2))
    dist, nb = cKDTree(P).query(P, k=k + 1)
    sigma = float(np.median(dist[:, k]))
    src = np.repeat(np.arange(n), k)
    dst = nb[:, 1:].reshape(-1)
    d = dist[:, 1:].reshape(-1)
    lo = np.minimum(src, dst).astype(np.int64)
    hi = np.maximum(src, dst).astype(np.int64)
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    w = np.exp(-(d[first] ** 2) / sigma ** 2)
    return from_edges(n, lo[first], hi[first], w)


def uniform(n, seed, lo=-1.0, hi=1.0):
    return _rng(seed).uniform(lo, hi, n)


def normal(n, seed):
    return _rng(seed).standard_normal(n)


def rhs(Q, xstar):
    """b = Q x* (consistent by construction), via a library sparse product."""
    n = int(Q["n"])
    A = _sp.csr_matrix((Q["val"], Q["col"], Q["row_ptr"]), shape=(n, n))
    return A @ np.asarray(xstar, np.float64)


def nnz(Q):
    return int(Q["row_ptr"][-1])


def workload(name, seed=None):
    """The named workloads used by tests and the benchmark: returns (Q, b, xstar)."""
    if name == "poisson2d_64":
        Q = poisson2d(64)
        xs = uniform(Q["n"], 1 if seed is None else seed)
    elif name == "poisson3d_256":
        Q = poisson3d(256)
        xs = normal(Q["n"], 2 if seed is None else seed)
    elif name.startswith("poisson3d_"):
        Q = poisson3d(int(name.split("_")[1]))
        xs = normal(Q["n"], 2 if seed is None else seed)
    elif name.startswith("poisson2d_"):
        Q = poisson2d(int(name.split("_")[1]))
        xs = uniform(Q["n"], 1 if seed is None else seed)
    elif name.startswith("chunglu_"):
        n = int(name.split("_")[1])
        Q = chung_lu_laplacian(n, seed=3 if seed is None else seed)
        xs = uniform(n, 3 if seed is None else seed + 1000)
    elif name.startswith("rgg_"):
        n = int(name.split("_")[1])
        Q = rgg_knn_laplacian(n, seed=4 if seed is None else seed)
        xs = uniform(n, 4 if seed is None else seed + 1000)
    else:
        raise KeyError(name)
    return Q, rhs(Q, xs), xs


def _log_uniform_int(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size)).astype(np.int64)


def batch_mix(count, seed=4, pool=48, side=(32, 1024), rgg_n=(1000, 500000), max_rhs=4):
    """Independent systems shaped like the batched workload: half 2-D Poisson
    grids with side log-uniform in ``side``, half k-NN random-geometric-graph
    Laplacians with n log-uniform in ``rgg_n``, each with 1..max_rhs
    right-hand sides b = Q x*, x* ~ U(-1, 1).

    To bound the generation time, the matrices come from a pool of ``pool``
    distinct ones (half of each kind, sizes drawn as above); every system picks
    one of its kind at random and draws its own x*.  Returns a list of
    ``(pool_index, nrhs, seeds)`` and the pool (a list of CSR dicts), so that
    callers can share device copies of pooled matrices.
    """
    rng = _rng(seed)
    half = max(1, pool // 2)
    sides = _log_uniform_int(rng, side[0], side[1] + 1, half)
    ns = _log_uniform_int(rng, rgg_n[0], rgg_n[1] + 1, half)
    mats = [poisson2d(int(s)) for s in sides]
    mats += [rgg_knn_laplacian(int(n), seed=seed * 100003 + k) for k, n in enumerate(ns)]
    systems = []
    for k in range(count):
        kind = k % 2
        j = int(rng.integers(0, half)) + kind * half
        nrhs = int(rng.integers(1, max_rhs + 1))
        systems.append((j, nrhs, [int(seed * 1000003 + 10 * k + r) for r in range(nrhs)]))
    return systems, mats


def served_mix(count, seed=5, pool=48, side3=(64, 192), frac3=0.2, **kw):
    """Requests shaped like the served workload: a fraction ``frac3`` are 3-D
    Poisson grids with side uniform in ``side3``; the rest follow
    ``batch_mix``.  Same pooled return form as ``batch_mix``."""
    systems, mats = batch_mix(count, seed=seed, pool=pool, **kw)
    rng = _rng(seed + 7)
    n3 = max(1, pool // 6)
    base = len(mats)
    mats += [poisson3d(int(s)) for s in rng.integers(side3[0], side3[1] + 1, n3)]
    out = []
    for j, nrhs, seeds in systems:
        if rng.random() < frac3:
            j = base + int(rng.integers(0, n3))
        out.append((j, nrhs, seeds))
    return out, mats


def mix_rhs(Q, seeds):
    """b (n x nrhs, column-major, flattened) for the x* seeds of one system."""
    return np.concatenate([rhs(Q, uniform(Q["n"], s)) for s in seeds])
