"""GPU checks of the locality ordering (reverse Cuthill-McKee renumbering,
AJ_REORDER_*).

Each renumbered row keeps its entries in the caller's order, so a row sums
exactly as before and only the grouping of the FP64 reductions changes: the
iterates, returned in the caller's row order, must follow the FP64 oracle to
the same 1e-10 as without renumbering.
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


def _fixed_parity(Q, B, T=200, x0=None, tol_rel=REL, **kw):
    nrhs = B.shape[1]
    ctx = aj.from_csr(Q, np.ascontiguousarray(B.T).reshape(-1), nrhs=nrhs)
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=T, x0=x0, **kw)
    X, infos = ctx.solve(per_rhs=True)
    X = X.reshape(nrhs, Q["n"])
    J = oracle.j_absrowsum(Q)
    for r in range(nrhs):
        xr0 = None if x0 is None else x0.reshape(nrhs, Q["n"])[r]
        ref = schedule.replay(Q, B[:, r], ctx.restart_log(r), T, J=J, x0=xr0)
        err = np.linalg.norm(X[r] - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= tol_rel, (r, err)
    return ctx


def _rhs(Q, nrhs, seed):
    return np.stack([synth.rhs(Q, synth.uniform(Q["n"], seed + r)) for r in range(nrhs)], axis=1)


def test_auto_renumbers_a_random_order_graph_and_keeps_parity():
    Q = synth.rgg_knn_laplacian(20000, seed=71)  # points in random order
    ctx = _fixed_parity(Q, _rhs(Q, 1, 5))
    reordered, before, after = ctx.order()
    assert reordered == 1 and after * 4 <= before


@pytest.mark.parametrize("nrhs", [1, 3])
def test_forced_rcm_with_x0_and_several_rhs(nrhs):
    Q = synth.rgg_knn_laplacian(3000, seed=72)
    B = _rhs(Q, nrhs, 9)
    x0 = np.ascontiguousarray(synth.uniform(Q["n"] * nrhs, 13))
    ctx = _fixed_parity(Q, B, x0=x0, reorder=aj.AJ_REORDER_RCM)
    assert ctx.order()[0] == 1


def test_natural_stencil_order_is_kept():
    Q = synth.poisson2d(200)  # n = 40000, rows gather within +-200
    ctx = aj.from_csr(Q, _rhs(Q, 1, 3)[:, 0])
    ctx.set(tol=1e-8)
    assert ctx.order()[0] == 0
    none = aj.from_csr(synth.rgg_knn_laplacian(20000, seed=71), np.ones(20000))
    none.set(reorder=aj.AJ_REORDER_NONE)
    assert none.order()[0] == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_renumbered_solve_reaches_tolerance(precision):
    Q = synth.rgg_knn_laplacian(30000, seed=73)
    b = synth.rhs(Q, synth.uniform(Q["n"], 17))
    ctx = aj.from_csr(Q, b, device="cuda")
    ctx.set(precision=precision, tol=1e-8, maxit=100000)
    assert ctx.order()[0] == 1
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK
    assert np.linalg.norm(b - oracle.spmv(Q, x)) <= 1e-8 * np.linalg.norm(b)


def test_resume_is_bit_identical_under_renumbering():
    Q = synth.rgg_knn_laplacian(3000, seed=74)
    b = synth.rhs(Q, synth.uniform(Q["n"], 19))
    full = aj.from_csr(Q, b)
    full.set(stop=aj.AJ_STOP_NONE, maxit=300, reorder=aj.AJ_REORDER_RCM)
    xf, _ = full.solve()
    part = aj.from_csr(Q, b)
    part.set(stop=aj.AJ_STOP_NONE, maxit=120, reorder=aj.AJ_REORDER_RCM)
    part.solve()
    blob = part.get_state()
    other = aj.from_csr(Q, b)
    other.set(stop=aj.AJ_STOP_NONE, maxit=300, reorder=aj.AJ_REORDER_RCM)
    other.set_state(blob)
    xr, _ = other.solve()
    np.testing.assert_array_equal(xr, xf)
    # a state saved in one row order is refused by a context in the other
    plain = aj.from_csr(Q, b)
    plain.set(stop=aj.AJ_STOP_NONE, maxit=300, reorder=aj.AJ_REORDER_NONE)
    with pytest.raises(aj.AJError):
        plain.set_state(blob)
