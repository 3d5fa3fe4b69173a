"""GPU checks of the block-diagonal J (eq. J-blkdiag, AJ_J_BLKDIAG).

aj_set builds every block J^{ii} = Q^{ii} + (sum_j ||Q^{ij}||_2) I and its
inverse on the device; the sweep applies the inverse across the lanes that
hold a block's rows.  The iterates must follow the FP64 oracle, which builds
the same blocks from the definition (dense SVD norms) and solves each block
with its Cholesky factor, to the 1e-10 of the diagonal-J path.
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


def _parity(Q, B, bs, T=200, tol_rel=REL, x0=None, **kw):
    nrhs = B.shape[1]
    ctx = _ctx(Q, B, j_policy=aj.AJ_J_BLKDIAG, j_block=bs, stop=aj.AJ_STOP_NONE, maxit=T, x0=x0, **kw)
    X, _ = ctx.solve(per_rhs=True)
    X = X.reshape(nrhs, Q["n"])
    Jb = oracle.j_blkdiag(Q, bs)
    for r in range(nrhs):
        xr0 = None if x0 is None else x0.reshape(nrhs, Q["n"])[r]
        ref = schedule.replay(Q, B[:, r], ctx.restart_log(r), T, Jblk=Jb, x0=xr0,
                              precision="df64" if kw.get("precision") == "df64" else "fp64")
        err = np.linalg.norm(X[r] - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= tol_rel, (r, err)
    return ctx, X


def _graph_with_components():
    # a Chung-Lu Laplacian (isolated vertices, small components) plus a few
    # 2-vertex components placed wholly inside blocks: singular blocks take J-diag
    Q = synth.chung_lu_laplacian(3001, seed=17, mean_degree=6.0)
    n = Q["n"]
    rp, ci, v = Q["row_ptr"], Q["col"], Q["val"]
    u, w, wt = [], [], []
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            if ci[p] > i:
                u.append(i), w.append(int(ci[p])), wt.append(-float(v[p]))
    keep = [(a, b, c) for a, b, c in zip(u, w, wt) if not (a < 80 or b < 80)]
    extra = [(8 * k, 8 * k + 1, 1.0) for k in range(10)]
    E = keep + extra
    return synth.from_edges(n, [e[0] for e in E], [e[1] for e in E], [e[2] for e in E])


@pytest.mark.parametrize("bs", [2, 4, 8])
@pytest.mark.parametrize("case", ["poisson2d_64", "poisson3d_13", "graph"])
def test_blkdiag_fp64_200_iterations_match_oracle(case, bs):
    if case == "graph":
        Q = _graph_with_components()
    elif case == "poisson3d_13":
        Q = synth.poisson3d(13)  # 2197 rows: a ragged last block for bs = 2, 4, 8
    else:
        Q, _, _ = synth.workload(case)
    B = _rhs(Q, seed=5)
    for fmt in (aj.AJ_FMT_CSR, aj.AJ_FMT_AUTO):
        _parity(Q, B, bs, format=fmt)


@pytest.mark.parametrize("nrhs", [2, 3, 4])
def test_blkdiag_several_rhs_with_x0(nrhs):
    Q = synth.rgg_knn_laplacian(2500, seed=9)
    B = _rhs(Q, nrhs=nrhs, seed=21)
    x0 = synth.uniform(Q["n"] * nrhs, 77)
    for bs in (4, 8):
        _parity(Q, B, bs, T=150, x0=x0)


@pytest.mark.parametrize("form", [aj.AJ_SWEEP_LAZY, aj.AJ_SWEEP_STORED, aj.AJ_SWEEP_DELTA, aj.AJ_SWEEP_Y])
def test_blkdiag_sweep_forms(form):
    Q = synth.poisson3d(11)
    B = _rhs(Q, seed=2)
    _parity(Q, B, 4, sweep_form=form)


def test_blkdiag_df64_matches_oracle():
    Q = synth.poisson2d(45)
    _parity(Q, _rhs(Q, seed=8), 4, precision="df64")


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32_ir", "bf16_ir"])
def test_blkdiag_solves_to_tolerance(precision):
    Q = synth.poisson3d(24)
    b = _rhs(Q, seed=4)[:, 0]
    for bs in (2, 8):
        c = _ctx(Q, b, j_policy=aj.AJ_J_BLKDIAG, j_block=bs, precision=precision, tol=1e-8, maxit=40000)
        x, info = c.solve()
        assert info["status"] == aj.AJ_OK
        r = b - oracle.spmv(Q, x)
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b)


def test_blkdiag_stencil_equals_csr_bitwise():
    Q = synth.poisson3d(19)
    B = _rhs(Q, nrhs=2, seed=6)
    kw = dict(j_policy=aj.AJ_J_BLKDIAG, j_block=4, tol=1e-9, maxit=40000, grid_ctas=5)
    for prec in ("fp64", "fp32_ir"):
        cs = _ctx(Q, B, format=aj.AJ_FMT_STENCIL, precision=prec, **kw)
        cc = _ctx(Q, B, format=aj.AJ_FMT_CSR, precision=prec, **kw)
        assert cs.format()[0] == aj.AJ_FMT_STENCIL and cc.format()[0] == aj.AJ_FMT_CSR
        xs, i_s = cs.solve(per_rhs=True)
        xc, i_c = cc.solve(per_rhs=True)
        np.testing.assert_array_equal(xs, xc)
        assert [i["iters"] for i in i_s] == [i["iters"] for i in i_c]


def test_block_of_one_is_j_diag_bitwise():
    Q = synth.chung_lu_laplacian(5000, seed=3, mean_degree=8.0)
    b = _rhs(Q, seed=1)
    c1 = _ctx(Q, b, j_policy=aj.AJ_J_BLKDIAG, j_block=1, stop=aj.AJ_STOP_NONE, maxit=120)
    c2 = _ctx(Q, b, j_policy=aj.AJ_J_ABSROWSUM, stop=aj.AJ_STOP_NONE, maxit=120)
    np.testing.assert_array_equal(c1.solve()[0], c2.solve()[0])


def test_blkdiag_batched_members_equal_solo():
    rng = np.random.default_rng(3)
    mix = []
    for k in range(8):
        Q = synth.poisson2d(int(rng.integers(6, 50))) if k % 2 else synth.rgg_knn_laplacian(
            int(rng.integers(300, 2500)), seed=300 + k)
        mix.append((Q, _rhs(Q, nrhs=int(rng.integers(1, 5)), seed=40 * k)))
    kw = dict(j_policy=aj.AJ_J_BLKDIAG, tol=1e-8, maxit=40000)
    for prec in ("fp64", "fp32_ir"):
        ctxs = [_ctx(Q, B, precision=prec, j_block=(2, 4, 8)[k % 3], grid_ctas=1 + k % 3, **kw)
                for k, (Q, B) in enumerate(mix)]
        outs = [np.empty(Q["n"] * B.shape[1]) for Q, B in mix]
        infos = aj.solve_batch(ctxs, outs)
        for k, ((Q, B), o, inf) in enumerate(zip(mix, outs, infos)):
            solo = _ctx(Q, B, precision=prec, j_block=(2, 4, 8)[k % 3], grid_ctas=1 + k % 3, **kw)
            xs, sinf = solo.solve()
            assert inf["status"] == sinf["status"] == aj.AJ_OK
            assert inf["iters"] == sinf["iters"]
            np.testing.assert_array_equal(o, xs)


def test_blkdiag_rejects_what_it_cannot_do():
    Q = synth.poisson2d(30)
    b = _rhs(Q)
    for kw in (dict(j_block=3), dict(j_block=16), dict(format=aj.AJ_FMT_SELL),
               dict(reorder=aj.AJ_REORDER_RCM)):
        with pytest.raises(RuntimeError):
            _ctx(Q, b, j_policy=aj.AJ_J_BLKDIAG, **kw)
    # rows longer than 1024 entries
    star = synth.from_edges(1500, [0] * 1499, list(range(1, 1500)), [1.0] * 1499)
    with pytest.raises(RuntimeError):
        _ctx(star, _rhs(star), j_policy=aj.AJ_J_BLKDIAG)
    # a random-order graph keeps the caller's order under AUTO
    G = synth.rgg_knn_laplacian(40000, seed=2)
    c = _ctx(G, _rhs(G), j_policy=aj.AJ_J_BLKDIAG, precision="fp32_ir")
    assert c.order()[0] == 0 and c.format()[0] == aj.AJ_FMT_CSR
