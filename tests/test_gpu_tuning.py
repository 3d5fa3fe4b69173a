"""The autotuner's axes against the oracle: SELL slice height C (rows per
warp step, 32 / C lanes per row), sorting window, long-row threshold and CTAs
per SM.  Every configuration the tuner can pick is also reachable by hand,
and each must follow the FP64 oracle's iterates (1e-10 after 200 iterations,
the restart schedule checked against Algorithm alg-apg-re); the tuner's
choice is reported by aj_get_tuning and cached per matrix shape.
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
FORMS = {"stored": aj.AJ_SWEEP_STORED, "lazy": aj.AJ_SWEEP_LAZY, "y": aj.AJ_SWEEP_Y}


def _graph(n=20000, seed=31):
    Q = synth.chung_lu_laplacian(n, seed=seed, mean_degree=16.0)
    return Q, synth.rhs(Q, synth.uniform(n, seed + 1))


def _parity(Q, b, T=200, precision="fp64", **kw):
    ctx = aj.from_csr(Q, b)
    ctx.set(precision=precision, stop=aj.AJ_STOP_NONE, maxit=T, **kw)
    x, info = ctx.solve()
    assert info["iters"] == T
    ref = schedule.replay(Q, b, ctx.restart_log(), T, J=oracle.j_absrowsum(Q),
                          precision="df64" if precision == "df64" else "fp64")
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= REL, err
    return ctx


@pytest.mark.parametrize("form", ["stored", "lazy", "y"])
@pytest.mark.parametrize("C", [32, 16, 8])
def test_sell_slice_heights_match_oracle(C, form):
    Q, b = _graph()
    assert np.diff(Q["row_ptr"]).max() > 64  # long rows in their bucket too
    ctx = _parity(Q, b, format=aj.AJ_FMT_SELL, sell_c=C, sweep_form=FORMS[form])
    t = ctx.tuning()
    assert t["format"] == aj.AJ_FMT_SELL and t["sell_c"] == C
    assert t["lanes_per_row"] == 32 // C and t["rows_per_cta"] == 8 * C
    assert t["sweep_form"] == FORMS[form] and t["tuned"] == 0


@pytest.mark.parametrize("C", [16, 8])
def test_sell_slice_heights_df64_and_solves(C):
    Q, b = _graph(seed=41)
    _parity(Q, b, T=150, precision="df64", format=aj.AJ_FMT_SELL, sell_c=C)
    for precision in ("fp64", "fp32_ir", "bf16_ir"):
        ctx = aj.from_csr(Q, b)
        ctx.set(precision=precision, tol=1e-8, maxit=40000, format=aj.AJ_FMT_SELL, sell_c=C)
        x, info = ctx.solve()
        assert info["status"] == aj.AJ_OK
        assert np.linalg.norm(b - oracle.spmv(Q, x)) <= 1e-8 * np.linalg.norm(b)


def test_several_rhs_keep_slices_of_32():
    Q, b = _graph(n=5000, seed=51)
    B = np.stack([b, synth.rhs(Q, synth.uniform(Q["n"], 52))], axis=1)
    ctx = aj.from_csr(Q, np.ascontiguousarray(B.T).reshape(-1), nrhs=2)
    ctx.set(format=aj.AJ_FMT_SELL, sell_c=8, stop=aj.AJ_STOP_NONE, maxit=100)
    t = ctx.tuning()
    assert t["sell_c"] == 32 and t["lanes_per_row"] == 2


def test_bad_slice_height_refused():
    Q, b = _graph(n=3000, seed=61)
    ctx = aj.from_csr(Q, b)
    with pytest.raises(aj.AJError):
        ctx.set(format=aj.AJ_FMT_SELL, sell_c=12)


def test_autotuner_choice_is_legal_cached_and_follows_the_oracle():
    # long-tailed rows and n >= 65536: AUTO times the candidates
    Q, b = _graph(n=100000, seed=71)
    ctx = aj.from_csr(Q, b)
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=100)
    t = ctx.tuning()
    assert t["tuned"] == 1
    assert t["format"] in (aj.AJ_FMT_CSR, aj.AJ_FMT_SELL)
    if t["format"] == aj.AJ_FMT_SELL:
        assert t["sell_c"] in (8, 16, 32) and t["sell_sigma"] in (256, 4096) and t["sell_lmax"] in (64, 256)
    assert 1 <= t["ctas_per_sm"] and t["grid"] >= 1 and t["threads_per_cta"] == 256
    # the same matrix again: the cached tuple
    ctx2 = aj.from_csr(Q, b)
    ctx2.set(stop=aj.AJ_STOP_NONE, maxit=100)
    assert ctx2.tuning() == t
    x, info = ctx.solve()
    ref = schedule.replay(Q, b, ctx.restart_log(), 100, J=oracle.j_absrowsum(Q))
    assert np.linalg.norm(x - ref["x"]) <= REL * np.linalg.norm(ref["x"])
    # the tuned run solves to tolerance
    ctx.set(tol=1e-8, maxit=20000)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK
    assert np.linalg.norm(b - oracle.spmv(Q, x)) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("C", [16, 8])
def test_batched_members_with_split_slices_equal_solo(C):
    Qa, ba = _graph(n=8000, seed=81)
    Qb, bb = _graph(n=12000, seed=83)
    kw = dict(format=aj.AJ_FMT_SELL, sell_c=C, tol=1e-8, maxit=20000, grid_ctas=3)
    ca = aj.from_csr(Qa, ba)
    ca.set(**kw)
    cb = aj.from_csr(Qb, bb)
    cb.set(**kw)
    xa, xb = np.empty(Qa["n"]), np.empty(Qb["n"])
    infos = aj.solve_batch([ca, cb], [xa, xb])
    for Q, b, x, inf in ((Qa, ba, xa, infos[0]), (Qb, bb, xb, infos[1])):
        solo = aj.from_csr(Q, b)
        solo.set(**kw)
        xs, sinf = solo.solve()
        assert inf["status"] == sinf["status"] == aj.AJ_OK and inf["iters"] == sinf["iters"]
        np.testing.assert_array_equal(x, xs)
