"""GPU checks of the SELL-C-sigma format (C = 32, sigma-sorted slices, a
warp-per-row bucket for long rows) and of the format autotuner.

Entries keep their CSR order inside every row, so a row sums in the same
order as in CSR; only the per-CTA reduction order differs.  The iterates
therefore match the FP64 oracle to the same 1e-10 as the CSR path.
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


def _fixed(Q, b, T, **kw):
    ctx = aj.from_csr(Q, b)
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=T, **kw)
    x, info = ctx.solve()
    return ctx, x, info


def _parity(Q, b, T, tol_rel=REL, **kw):
    ctx, x, info = _fixed(Q, b, T, **kw)
    fmt = ctx.format()
    # the oracle with the GPU's restart schedule, checked against the rule
    ref = schedule.replay(Q, b, ctx.restart_log(), T, J=oracle.j_absrowsum(Q),
                          precision="df64" if kw.get("precision") == "df64" else "fp64")
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= tol_rel, (err, fmt)
    return ctx, x, fmt


def _chunglu(n, seed, deg=16.0):
    Q = synth.chung_lu_laplacian(n, seed=seed, mean_degree=deg)
    b = synth.rhs(Q, synth.uniform(n, seed + 1))
    return Q, b


@pytest.mark.parametrize("sigma,lmax", [(1, 64), (256, 64), (4096, 64), (256, 16), (32, 100000)])
def test_sell_fp64_matches_oracle_on_power_law_rows(sigma, lmax):
    Q, b = _chunglu(20000, 31)
    lens = np.diff(Q["row_ptr"])
    assert lens.max() > 64 and (lens == 0).any()
    ctx, x, fmt = _parity(Q, b, 150, format=aj.AJ_FMT_SELL, sell_sigma=sigma, sell_lmax=lmax)
    assert fmt[:3] == (aj.AJ_FMT_SELL, sigma, lmax)
    assert fmt[3] >= 1.0


def test_sell_on_stencils_with_ragged_tail():
    Q, b, xs = synth.workload("poisson3d_13")  # n = 2197: ragged last slice and tile
    ctx, x, fmt = _parity(Q, b, 120, format=aj.AJ_FMT_SELL)
    assert fmt[0] == aj.AJ_FMT_SELL


@pytest.mark.parametrize("precision", ["df64", "fp32_ir", "bf16_ir"])
def test_sell_other_precisions(precision):
    if precision == "bf16_ir":
        Q, b, xs = synth.workload("poisson2d_64")
    else:
        Q, b = _chunglu(20000, 41)
    if precision == "df64":
        _parity(Q, b, 150, format=aj.AJ_FMT_SELL, precision=precision)
    ctx = aj.from_csr(Q, b)
    ctx.set(precision=precision, tol=1e-8, maxit=40000, format=aj.AJ_FMT_SELL)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK
    assert np.linalg.norm(b - oracle.spmv(Q, x)) <= 1e-8 * np.linalg.norm(b)


def test_sell_and_csr_iterates_agree():
    Q, b = _chunglu(30000, 51)
    _, xc, _ = _fixed(Q, b, 100, format=aj.AJ_FMT_CSR, restart=0)
    _, xs, _ = _fixed(Q, b, 100, format=aj.AJ_FMT_SELL, restart=0)
    assert np.linalg.norm(xc - xs) <= 1e-12 * np.linalg.norm(xc)


def test_autotuner_picks_a_format_and_solves():
    Q, b = _chunglu(1 << 17, 61)
    ctx = aj.from_csr(Q, b, device="cuda")
    ctx.set(tol=1e-8, maxit=40000, precision="fp32_ir")
    fmt = ctx.format()
    assert fmt[0] in (aj.AJ_FMT_CSR, aj.AJ_FMT_SELL)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK
    assert np.linalg.norm(b - oracle.spmv(Q, x)) <= 1e-8 * np.linalg.norm(b)
    # the choice is cached per shape: a second context gets it without timing
    ctx2 = aj.from_csr(Q, b, device="cuda")
    ctx2.set(tol=1e-8, maxit=40000, precision="fp32_ir")
    assert ctx2.format()[:3] == fmt[:3]
    # grid stencils get the stencil format, never SELL; their rows are uniform,
    # so with the stencil format off they keep CSR without timing
    Qp, bp, _ = synth.workload("poisson3d_64")
    c3 = aj.from_csr(Qp, bp, device="cuda")
    c3.set(tol=1e-8)
    assert c3.format()[0] == aj.AJ_FMT_STENCIL
    Qp["val"] = Qp["val"] * 1.0
    Qp["val"][0] = 6.5  # row 0's diagonal: no longer one diagonal value
    c4 = aj.from_csr(Qp, bp, device="cuda")
    c4.set(tol=1e-8)
    assert c4.format()[0] == aj.AJ_FMT_CSR
