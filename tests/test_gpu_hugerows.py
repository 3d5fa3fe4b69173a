"""Rows of more than 4096 entries against the oracle.

In the SELL-C-sigma format such rows are summed by a whole CTA (one row per
tile, threads striding over its entries, then a fixed tree), and rows of 33
to 4096 entries by a whole warp.  The hubs of power-law graphs and the dense
rows of the Section 4.1 system take that path, and so does the 8.4M-vertex
Chung-Lu graph of the benchmark (its largest row has over 11,000 entries).
"""
import numpy as np
import pytest

import oracle
from oracle import schedule
import synth
from stepcheck import one_step, state_parts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402

REL = 1e-10
HUGE = 4096  # rows above this many entries are summed by a whole CTA in SELL


def _hub_graph():
    # a Chung-Lu Laplacian (n = 60,000, mean degree 8) with two planted hubs:
    # rows of 6006 and 6575 entries, beside ordinary rows of up to ~700
    Q = synth.chung_lu_laplacian(60000, seed=91, mean_degree=8.0)
    return synth.with_hubs(Q, [5, 30001], 6000, seed=92)


def _parity(Q, B, T, **kw):
    nrhs = B.shape[1]
    ctx = aj.from_csr(Q, np.ascontiguousarray(B.T).reshape(-1), nrhs=nrhs)
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=T, **kw)
    X, infos = ctx.solve(per_rhs=True)
    X = X.reshape(nrhs, Q["n"])
    J = oracle.j_absrowsum(Q)
    for r in range(nrhs):
        assert infos[r]["iters"] == T
        ref = schedule.replay(Q, B[:, r], ctx.restart_log(r), T, J=J)
        err = np.linalg.norm(X[r] - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= REL, (r, err)
    return ctx


@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("fmt", ["sell", "auto"])
def test_hub_rows_200_iterations_match_oracle(nrhs, fmt):
    Q = _hub_graph()
    lens = np.diff(Q["row_ptr"])
    assert (lens > HUGE).sum() == 2
    B = np.stack([synth.rhs(Q, synth.uniform(Q["n"], 93 + r)) for r in range(nrhs)], axis=1)
    kw = dict(format=aj.AJ_FMT_SELL) if fmt == "sell" else {}
    ctx = _parity(Q, B, 200, **kw)
    if fmt == "sell":
        assert ctx.format()[0] == aj.AJ_FMT_SELL  # AUTO may time CSR (warp-summed hubs) faster


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_dense_rows_of_the_section_4_1_system(precision):
    # n = 4200 > 4096: every row is a CTA-summed row; AUTO takes SELL for few dense rows
    n = 4200
    Q = synth.sdd(n)
    b = np.ones(n)
    ctx = aj.from_csr(Q, b)
    T = 100
    ctx.set(precision=precision, stop=aj.AJ_STOP_NONE, maxit=T)
    assert ctx.format()[0] == aj.AJ_FMT_SELL
    x, info = ctx.solve()
    ref = schedule.replay(Q, b, ctx.restart_log(), T, J=oracle.j_absrowsum(Q), precision=precision)
    assert np.linalg.norm(x - ref["x"]) <= REL * np.linalg.norm(ref["x"])


def test_fullsize_graph_step_matches_oracle_step():
    """The benchmark's graph: Chung-Lu, n = 8,388,608, nnz = 142,568,568, in the
    format AUTO picks (SELL, with CTA-summed hub rows).  One GPU iteration from
    the GPU's own state against one oracle iteration, 1e-12."""
    Q, b, _ = synth.workload("chunglu_8388608")
    n = Q["n"]
    assert np.diff(Q["row_ptr"]).max() > HUGE
    T = 30
    ctx = aj.from_csr(Q, b, device="cuda")
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=T)
    assert ctx.format()[0] == aj.AJ_FMT_SELL and ctx.order()[0] == 0
    ctx.solve(out=torch.empty(n, dtype=torch.float64, device="cuda"))
    blob = ctx.get_state()
    st = state_parts(blob, n)
    assert st["t"] == T
    ctx2 = aj.from_csr(Q, b, device="cuda")
    ctx2.set(stop=aj.AJ_STOP_NONE, maxit=T + 1)
    ctx2.set_state(blob)
    x_next, info = ctx2.solve()
    assert info["iters"] == T + 1
    ref = one_step(Q, b, oracle.j_absrowsum(Q), st, (T + 1) in ctx2.restart_log())
    err = np.linalg.norm(x_next - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err
