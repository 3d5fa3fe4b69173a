"""GPU checks of the constant-coefficient stencil format (AJ_FMT_STENCIL).

For the grid Laplacians of Sec. 4 the fused sweep computes each row's columns
and values from the row index instead of loading them.  It visits the same
columns in the same ascending order with the same (precision-rounded) values
as the CSR rows, so every row sum, and with the same grid every reduction, is
the CSR one bit for bit: the iterates of the two formats must be identical in
every precision and sweep form.  Detection checks every row on the device, so
a matrix that differs anywhere keeps CSR.
"""
import numpy as np
import pytest

import oracle
from oracle import schedule
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402

REL = 1e-10


def _ctx(Q, B, **kw):
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    ctx = aj.from_csr(Q, np.ascontiguousarray(B.T).reshape(-1), nrhs=B.shape[1])
    ctx.set(**kw)
    return ctx


def _rhs(Q, nrhs=1, seed=0):
    return np.stack([synth.rhs(Q, synth.uniform(Q["n"], seed + r)) for r in range(nrhs)], axis=1)


def _pair(Q, B, **kw):
    """The same solve in the stencil format and in CSR: (x, info) of each."""
    cs = _ctx(Q, B, format=aj.AJ_FMT_STENCIL, **kw)
    assert cs.format()[0] == aj.AJ_FMT_STENCIL
    cc = _ctx(Q, B, format=aj.AJ_FMT_CSR, **kw)
    assert cc.format()[0] == aj.AJ_FMT_CSR
    xs, inf_s = cs.solve(per_rhs=True)
    xc, inf_c = cc.solve(per_rhs=True)
    return (cs, xs, inf_s), (cc, xc, inf_c)


def _assert_same(a, b):
    (cs, xs, inf_s), (cc, xc, inf_c) = a, b
    np.testing.assert_array_equal(xs, xc)
    for i, j in zip(inf_s, inf_c):
        assert i["iters"] == j["iters"] and i["restarts"] == j["restarts"]
        assert i["status"] == j["status"]
    for r in range(len(inf_s)):
        assert cs.restart_log(r) == cc.restart_log(r)


@pytest.mark.parametrize("name,dim", [("2d", 2), ("3d", 3)])
def test_auto_detects_grid_stencils(name, dim):
    Q = synth.poisson2d(37) if dim == 2 else synth.poisson3d(13)
    c = _ctx(Q, _rhs(Q))
    f = c.format()
    assert f[0] == aj.AJ_FMT_STENCIL and f[3] == 0.0
    c2 = _ctx(Q, _rhs(Q), format=aj.AJ_FMT_CSR)
    assert c2.format()[0] == aj.AJ_FMT_CSR


def test_auto_rule_per_precision_and_form():
    # AUTO keeps CSR where the stencil format measured slower: FP64 with
    # several right-hand sides or in the lazy form
    Q = synth.poisson2d(45)
    expect = [(dict(), 1, aj.AJ_FMT_STENCIL),
              (dict(sweep_form=aj.AJ_SWEEP_STORED), 1, aj.AJ_FMT_STENCIL),
              (dict(sweep_form=aj.AJ_SWEEP_LAZY), 1, aj.AJ_FMT_CSR),
              (dict(), 2, aj.AJ_FMT_CSR),
              (dict(precision="df64"), 3, aj.AJ_FMT_STENCIL),
              (dict(precision="fp32_ir"), 4, aj.AJ_FMT_STENCIL),
              (dict(precision="bf16_ir", sweep_form=aj.AJ_SWEEP_LAZY), 1, aj.AJ_FMT_STENCIL)]
    for kw, nrhs, fmt in expect:
        assert _ctx(Q, _rhs(Q, nrhs=nrhs), **kw).format()[0] == fmt, (kw, nrhs)
    assert _ctx(Q, _rhs(Q, nrhs=2), format=aj.AJ_FMT_STENCIL).format()[0] == aj.AJ_FMT_STENCIL


@pytest.mark.parametrize("precision,form", [
    ("fp64", aj.AJ_SWEEP_DELTA), ("fp64", aj.AJ_SWEEP_STORED), ("fp64", aj.AJ_SWEEP_LAZY),
    ("fp64", aj.AJ_SWEEP_Y), ("df64", aj.AJ_SWEEP_STORED), ("df64", aj.AJ_SWEEP_LAZY),
    ("df64", aj.AJ_SWEEP_Y), ("fp32_ir", aj.AJ_SWEEP_LAZY), ("fp32_ir", aj.AJ_SWEEP_STORED),
    ("fp32_ir", aj.AJ_SWEEP_Y), ("bf16_ir", aj.AJ_SWEEP_LAZY), ("bf16_ir", aj.AJ_SWEEP_STORED),
    ("bf16_ir", aj.AJ_SWEEP_Y)])
def test_stencil_iterates_bitwise_equal_csr(precision, form):
    # 3-D 23^3: 12167 rows, 47 full tiles and a ragged one
    Q = synth.poisson3d(23)
    B = _rhs(Q, seed=7)
    for grid in (7, 0):
        a, b = _pair(Q, B, precision=precision, sweep_form=form, tol=1e-8, maxit=40000, grid_ctas=grid)
        _assert_same(a, b)
        assert a[2][0]["status"] == aj.AJ_OK and a[2][0]["relres"] <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "bf16_ir", "df64", "fp32_ir"])
@pytest.mark.parametrize("N,dim", [(37, 2), (5, 3), (3, 2)])
def test_staged_stencil_grids_bitwise_equal_csr(precision, N, dim):
    # the explicit-y stencil sweep whose gathers are staged in shared memory
    # (FP64 and BF16 values; the other two run unstaged): odd sides, so the
    # +-N segments start off a 16-byte boundary; a 2-D grid (no +-N^2
    # segments); ragged last tiles; and a grid smaller than one tile
    Q = synth.poisson2d(N) if dim == 2 else synth.poisson3d(N)
    B = _rhs(Q, seed=13)
    for grid in (3, 0):
        a, b = _pair(Q, B, precision=precision, sweep_form=aj.AJ_SWEEP_Y, tol=1e-8, maxit=40000,
                     grid_ctas=grid)
        _assert_same(a, b)
        assert a[2][0]["status"] == aj.AJ_OK and a[2][0]["relres"] <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_stencil_multi_rhs_and_x0_bitwise_equal_csr(precision):
    Q = synth.poisson2d(53)
    B = _rhs(Q, nrhs=3, seed=11)
    x0 = synth.uniform(Q["n"] * 3, 99)
    for nrhs in (2, 3):
        a, b = _pair(Q, B[:, :nrhs], precision=precision, tol=1e-8, maxit=40000,
                     x0=np.ascontiguousarray(x0[:Q["n"] * nrhs]))
        _assert_same(a, b)


def test_stencil_fixed_200_iterations_match_oracle():
    # the small 2-D Poisson 64 x 64 system, 200 fixed iterations
    Q, b, _ = synth.workload("poisson2d_64")
    c = _ctx(Q, b, stop=aj.AJ_STOP_NONE, maxit=200)
    assert c.format()[0] == aj.AJ_FMT_STENCIL
    x, _ = c.solve()
    J = oracle.j_absrowsum(Q)
    ref = schedule.replay(Q, b, c.restart_log(), 200, J=J)
    assert np.linalg.norm(x - ref["x"]) <= REL * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("make", [lambda: synth.poisson2d(2), lambda: synth.poisson3d(2),
                                  lambda: synth.poisson2d(8), lambda: synth.poisson3d(4)])
def test_small_and_ambiguous_grids(make):
    # n = 4 and 8 are the smallest grids; n = 64 is both 8^2 and 4^3 (told apart by nnz)
    Q = make()
    B = _rhs(Q, seed=3)
    a, b = _pair(Q, B, tol=1e-10, maxit=20000)
    _assert_same(a, b)


def _perturbed(Q, k):
    """Q with the symmetric pair of entries k, k' scaled (still SPSD, SDD)."""
    Q = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in Q.items()}
    rp, ci, val = Q["row_ptr"], Q["col"], Q["val"]
    i = int(np.searchsorted(rp, k, side="right") - 1)
    j = int(ci[k])
    assert i != j
    val[k] *= 0.5
    kk = int(rp[j] + np.nonzero(ci[rp[j]:rp[j + 1]] == i)[0][0])
    val[kk] *= 0.5
    return Q


def test_other_matrices_keep_csr():
    Q = synth.poisson3d(11)
    cases = [_perturbed(Q, int(Q["row_ptr"][-1]) // 2 + 1)]
    # one row's entries out of ascending order
    Qs = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in Q.items()}
    r = Q["n"] // 3
    lo, hi = int(Qs["row_ptr"][r]), int(Qs["row_ptr"][r + 1])
    Qs["col"][lo:hi] = Qs["col"][lo:hi][::-1].copy()
    Qs["val"][lo:hi] = Qs["val"][lo:hi][::-1].copy()
    cases.append(Qs)
    # a scaled diagonal in one row
    Qd = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in Q.items()}
    d = int(Qd["row_ptr"][5] + np.nonzero(Qd["col"][Qd["row_ptr"][5]:Qd["row_ptr"][6]] == 5)[0][0])
    Qd["val"][d] = 6.5
    cases.append(Qd)
    cases.append(synth.chung_lu_laplacian(4096, seed=5, mean_degree=6.0))
    for M in cases:
        b = _rhs(M)
        c = _ctx(M, b, tol=1e-8, maxit=40000)
        assert c.format()[0] != aj.AJ_FMT_STENCIL
        x, info = c.solve()
        assert info["status"] == aj.AJ_OK
        with pytest.raises(RuntimeError):
            _ctx(M, b, format=aj.AJ_FMT_STENCIL)


def test_explicit_stencil_with_renumbering_is_refused():
    Q = synth.poisson2d(40)
    with pytest.raises(RuntimeError):
        _ctx(Q, _rhs(Q), format=aj.AJ_FMT_STENCIL, reorder=aj.AJ_REORDER_RCM)
    c = _ctx(Q, _rhs(Q), reorder=aj.AJ_REORDER_RCM)
    assert c.order()[0] == 1 and c.format()[0] == aj.AJ_FMT_CSR


@pytest.mark.parametrize("precision,form", [("fp64", "auto"), ("fp32_ir", "lazy"), ("fp32_ir", "y")])
def test_batched_stencil_members_equal_csr(precision, form):
    # both formats in the same sweep form (AUTO gives one-RHS FP32 members in
    # the stencil format the explicit-y form, on CSR the lazy one)
    sf = {"auto": aj.AJ_SWEEP_AUTO, "lazy": aj.AJ_SWEEP_LAZY, "y": aj.AJ_SWEEP_Y}[form]
    rng = np.random.default_rng(5)
    mix = []
    for k in range(10):
        Q = synth.poisson2d(int(rng.integers(5, 60))) if k % 2 else synth.poisson3d(int(rng.integers(3, 16)))
        mix.append((Q, _rhs(Q, nrhs=int(rng.integers(1, 5)), seed=50 * k)))
    out = {}
    for fmt in (aj.AJ_FMT_STENCIL, aj.AJ_FMT_CSR):
        ctxs = [_ctx(Q, B, format=fmt, precision=precision, tol=1e-8, maxit=40000, grid_ctas=1 + k % 3,
                     sweep_form=sf)
                for k, (Q, B) in enumerate(mix)]
        outs = [np.empty(Q["n"] * B.shape[1]) for Q, B in mix]
        infos = aj.solve_batch(ctxs, outs)
        out[fmt] = (outs, infos)
    for xs, xc, i, j in zip(out[aj.AJ_FMT_STENCIL][0], out[aj.AJ_FMT_CSR][0],
                            out[aj.AJ_FMT_STENCIL][1], out[aj.AJ_FMT_CSR][1]):
        np.testing.assert_array_equal(xs, xc)
        assert i["iters"] == j["iters"] and i["status"] == j["status"] == aj.AJ_OK
