"""Full-size checks on the 3-D 7-point Poisson system on a 256^3 grid
(n = 16,777,216, nnz = 117,047,296), in the launch configuration the
benchmark times.  The oracle cannot run thousands of iterations at this size,
so the GPU's iterate x^{T+1} is checked against one oracle step taken from
the GPU's own x^T, x^{T-1} and beta_T (read from the solver state), and every
solve's residual is recomputed with the oracle's FP64 SpMV.
"""
import numpy as np
import pytest

import oracle
import synth
from stepcheck import one_step, state_parts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402

_W = {}


def workload():
    if "w" not in _W:
        _W["w"] = synth.workload("poisson3d_256")
    return _W["w"]


@pytest.mark.parametrize("fmt", ["csr", "stencil"])
def test_fullsize_step_matches_oracle_step(fmt):
    # CSR is the benchmark's configuration; AUTO takes the stencil format here
    Q, b, xs = workload()
    n = Q["n"]
    T = 40
    F = aj.AJ_FMT_CSR if fmt == "csr" else aj.AJ_FMT_STENCIL
    ctx = aj.from_csr(Q, b, device="cuda")
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=T, format=F)
    assert ctx.format()[0] == F
    ctx.solve(out=torch.empty(n, dtype=torch.float64, device="cuda"))
    st = state_parts(ctx.get_state(), n)
    assert st["t"] == T
    ctx2 = aj.from_csr(Q, b, device="cuda")
    ctx2.set(stop=aj.AJ_STOP_NONE, maxit=T + 1, format=F)
    ctx2.set_state(ctx.get_state())
    x_next, info = ctx2.solve()
    assert info["iters"] == T + 1
    ref = one_step(Q, b, oracle.j_absrowsum(Q), st, (T + 1) in ctx2.restart_log())
    err = np.linalg.norm(x_next - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err


@pytest.mark.parametrize("precision,kw", [
    ("df64", {}), ("fp32_ir", {}), ("fp64", {}), ("bf16_ir", {}),
    ("fp64", dict(format=aj.AJ_FMT_CSR)), ("fp32_ir", dict(format=aj.AJ_FMT_CSR)),
    ("fp32_ir", dict(j_policy=aj.AJ_J_BLKDIAG, j_block=4)), ("fp64", dict(j_policy=aj.AJ_J_BLKDIAG, j_block=8))])
def test_fullsize_solve_reaches_1e8(precision, kw):
    Q, b, xs = workload()
    ctx = aj.from_csr(Q, b, device="cuda")
    ctx.set(precision=precision, tol=1e-8, maxit=30000, **kw)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK, info
    r = b - oracle.spmv(Q, x)
    rr = np.linalg.norm(r) / np.linalg.norm(b)
    assert rr <= 1e-8
    assert abs(rr - info["relres"]) <= 1e-3 * rr


@pytest.mark.parametrize("precision,form", [("fp64", "auto"), ("fp32_ir", "lazy"), ("fp32_ir", "y"),
                                            ("bf16_ir", "auto")])
def test_fullsize_stencil_equals_csr_bitwise(precision, form):
    # the stencil rows are the CSR rows' sums bit for bit, at the full size
    # too, in the same sweep form (AUTO gives FP32 values in the stencil
    # format the explicit-y form, on CSR the lazy one)
    Q, b, xs = workload()
    n = Q["n"]
    sf = {"auto": aj.AJ_SWEEP_AUTO, "lazy": aj.AJ_SWEEP_LAZY, "y": aj.AJ_SWEEP_Y}[form]
    out = {}
    for F in (aj.AJ_FMT_CSR, aj.AJ_FMT_STENCIL):
        c = aj.from_csr(Q, b, device="cuda")
        c.set(precision=precision, stop=aj.AJ_STOP_NONE, maxit=60, inner_tol=1e-30, format=F, sweep_form=sf)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        _, info = c.solve(out=x)
        out[F] = (x.cpu().numpy(), info["iters"])
        c.close()
    np.testing.assert_array_equal(out[aj.AJ_FMT_CSR][0], out[aj.AJ_FMT_STENCIL][0])
    assert out[aj.AJ_FMT_CSR][1] == out[aj.AJ_FMT_STENCIL][1]


def test_fullsize_pcg_reaches_1e8():
    Q, b, xs = workload()
    c = aj.from_csr(Q, b, device="cuda")
    c.set(tol=1e-8, maxit=5000)
    x, info = c.pcg_solve()
    assert info["status"] == aj.AJ_OK, info
    rr = np.linalg.norm(b - oracle.spmv(Q, x)) / np.linalg.norm(b)
    assert rr <= 1.01e-8 and abs(rr - info["relres"]) <= 1e-3 * rr
