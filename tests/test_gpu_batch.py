"""GPU checks of aj_solve_batch: many independent systems of different sizes
and right-hand-side counts in one persistent launch per right-hand-side count
(gangs of CTAs, each system with its own momentum, restart and stop state).

* A batch member whose grid_ctas is fixed computes exactly what aj_solve
  computes alone with the same grid_ctas: bitwise equal iterates.
* Without it every member still reaches its FP64-verified tolerance and
  matches the FP64 oracle's converged solution in the Q-norm.
* The mixed-precision (FP32 values, FP64 refinement) batch reaches 1e-8 on
  every system, and a member that runs out of iterations reports it without
  disturbing the others.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402


def _relres(Q, b, x):
    r = b - oracle.spmv(Q, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def _mix(count, seed=0, kinds=3):
    """A seeded mix of 2-D Poisson grids, k-NN graph Laplacians and Chung-Lu
    Laplacians (kinds = 1: Poisson only) with 1..4 right-hand sides each."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        kind = k % kinds
        if kind == 0:
            Q = synth.poisson2d(int(rng.integers(6, 48)))
        elif kind == 1:
            Q = synth.rgg_knn_laplacian(int(rng.integers(300, 3000)), seed=100 + k)
        else:
            Q = synth.chung_lu_laplacian(int(rng.integers(500, 4000)), seed=200 + k, mean_degree=6.0)
        nrhs = int(rng.integers(1, 5))
        n = Q["n"]
        B = np.stack([synth.rhs(Q, synth.uniform(n, 1000 * k + r)) for r in range(nrhs)], axis=1)
        out.append((Q, B))
    return out


def _ctx(Q, B, **kw):
    nrhs = B.shape[1]
    ctx = aj.from_csr(Q, np.ascontiguousarray(B.T).reshape(-1), nrhs=nrhs)
    ctx.set(**kw)
    return ctx


def _batch(ctxs, mix):
    outs = [np.empty(Q["n"] * B.shape[1]) for Q, B in mix]
    infos = aj.solve_batch(ctxs, outs)
    return [o.reshape(B.shape[1], Q["n"]).T for o, (Q, B) in zip(outs, mix)], infos


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_batch_member_equals_solo_with_same_gang(precision):
    mix = _mix(18, seed=1)
    kw = dict(precision=precision, tol=1e-9, maxit=20000)
    gangs = [1 + (k % 3) for k in range(len(mix))]
    ctxs = [_ctx(Q, B, grid_ctas=g, **kw) for (Q, B), g in zip(mix, gangs)]
    X, infos = _batch(ctxs, mix)
    for (Q, B), g, x, inf in zip(mix, gangs, X, infos):
        solo = _ctx(Q, B, grid_ctas=g, **kw)
        xs, sinf = solo.solve()
        xs = xs.reshape(B.shape[1], Q["n"]).T
        assert inf["status"] == aj.AJ_OK and sinf["status"] == aj.AJ_OK
        assert inf["iters"] == sinf["iters"]
        np.testing.assert_array_equal(x, xs)


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir", "bf16_ir"])
def test_batch_reaches_tolerance_and_matches_oracle(precision):
    # BF16 keeps the integer Poisson stencils exact; it rounds graph weights by
    # up to 2^-9 relative, which breaks their zero row sums, and the inner
    # solve on that perturbed matrix can diverge: Poisson systems only there.
    mix = _mix(30, seed=2, kinds=1 if precision == "bf16_ir" else 3)
    ctxs = [_ctx(Q, B, precision=precision, tol=1e-8, maxit=40000) for Q, B in mix]
    X, infos = _batch(ctxs, mix)
    for (Q, B), x, inf in zip(mix, X, infos):
        assert inf["status"] == aj.AJ_OK, inf
        for r in range(B.shape[1]):
            assert _relres(Q, B[:, r], x[:, r]) <= 1e-8
    # Q-norm error against the oracle's converged solution on a few members
    for k in (0, 1, 2):
        Q, B = mix[k]
        ref = oracle.solve(Q, B[:, 0], oracle.j_absrowsum(Q), tol=1e-12, maxit=200000)
        e = X[k][:, 0] - ref["x"]
        qe = math.sqrt(max(e @ oracle.spmv(Q, e), 0.0))
        qx = math.sqrt(ref["x"] @ oracle.spmv(Q, ref["x"]))
        assert qe <= 1e-6 * qx


def test_batch_member_out_of_iterations_does_not_disturb_others():
    mix = _mix(6, seed=3)
    ctxs = [_ctx(Q, B, tol=1e-8, maxit=(15 if k == 2 else 20000)) for k, (Q, B) in enumerate(mix)]
    X, infos = _batch(ctxs, mix)
    for k, inf in enumerate(infos):
        if k == 2:
            assert inf["status"] == aj.AJ_EMAXIT and inf["iters"] == 15
        else:
            assert inf["status"] == aj.AJ_OK


def test_batch_of_many_small_systems_uses_many_gangs():
    rng = np.random.default_rng(4)
    mix = []
    for k in range(160):
        Q = synth.poisson2d(int(rng.integers(4, 80)))
        n = Q["n"]
        mix.append((Q, synth.rhs(Q, synth.uniform(n, k))[:, None]))
    ctxs = [_ctx(Q, B, tol=1e-8, maxit=20000) for Q, B in mix]
    X, infos = _batch(ctxs, mix)
    for (Q, B), x, inf in zip(mix, X, infos):
        assert inf["status"] == aj.AJ_OK
        assert _relres(Q, B[:, 0], x[:, 0]) <= 1e-8


def test_batch_rejects_mixed_precisions_and_duplicates():
    Q = synth.poisson2d(8)
    b = synth.rhs(Q, synth.uniform(64, 1))
    c1 = _ctx(Q, b[:, None], precision="fp64")
    c2 = _ctx(Q, b[:, None], precision="fp32_ir")
    with pytest.raises(aj.AJError):
        aj.solve_batch([c1, c2], [np.empty(64), np.empty(64)])
    with pytest.raises(aj.AJError):
        aj.solve_batch([c1, c1], [np.empty(64), np.empty(64)])


@pytest.mark.parametrize("precision", ["fp32_ir", "fp64"])
def test_batch_of_mixed_sweep_forms_equals_solo(precision):
    # members of one precision whose sweep forms differ (SELL members take the
    # stored form under AUTO in FP32; FP64 members here name their form) run as
    # one lockstep batch per form, each member bit for bit its solo run
    mix = _mix(9, seed=9)
    kws = []
    for k in range(len(mix)):
        kw = dict(precision=precision, tol=1e-8, maxit=40000, grid_ctas=1 + k % 2)
        if precision == "fp32_ir":
            kw["format"] = aj.AJ_FMT_SELL if k % 3 == 0 else aj.AJ_FMT_CSR
        else:
            kw["sweep_form"] = (aj.AJ_SWEEP_DELTA, aj.AJ_SWEEP_STORED, aj.AJ_SWEEP_LAZY, aj.AJ_SWEEP_Y)[k % 4]
        kws.append(kw)
    ctxs = [_ctx(Q, B, **kw) for (Q, B), kw in zip(mix, kws)]
    X, infos = _batch(ctxs, mix)
    for (Q, B), kw, x, inf in zip(mix, kws, X, infos):
        solo = _ctx(Q, B, **kw)
        xs, sinf = solo.solve()
        xs = xs.reshape(B.shape[1], Q["n"]).T
        assert inf["status"] == sinf["status"] == aj.AJ_OK
        assert inf["iters"] == sinf["iters"]
        np.testing.assert_array_equal(x, xs)
