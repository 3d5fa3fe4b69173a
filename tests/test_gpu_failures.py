"""Failure detection without a GPU fault.

Each error path of the solver is driven from the host or by a bounded wait:
- AJ_EDIVERGED: J = L D with L half of lambda_max(D^-1/2 Q D^-1/2), so that
  S = J - Q is not PSD (the condition of Algorithm alg-jacobi fails) and the
  residual grows without bound; the kernel stops once it passes 1e8 times
  its starting value.
- AJ_ENONFINITE: a right-hand side near 1e200 whose squared norm overflows in
  the kernel's FP64 reduction.
- AJ_ETIMEOUT: one CTA withholds its first grid-barrier arrival
  (aj_test_barrier_stall) and the others' waits, limited to 2 ms, run out.
- AJ_ENOMEM: a device allocation made to fail on the host
  (aj_test_alloc_fail) inside aj_create and inside aj_set.
After each, the context (or a new one) solves normally.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402


def _poisson(N):
    Q, b, _ = synth.workload("poisson2d_%d" % N)
    return Q, b


def _ok_solve(ctx, Q, b):
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK
    assert np.linalg.norm(b - oracle.spmv(Q, x)) <= 1e-8 * np.linalg.norm(b)
    return x


@pytest.mark.parametrize("precision,form", [("fp64", "delta"), ("fp64", "y"), ("df64", "auto")])
def test_diverging_step_constant_is_detected(precision, form):
    N = 16
    Q, b = _poisson(N)
    lam = 1.0 + math.cos(math.pi / (N + 1))  # lambda_max(D^-1/2 Q D^-1/2), closed form
    L = 0.5 * lam
    ctx = aj.from_csr(Q, b)
    sf = {"delta": aj.AJ_SWEEP_DELTA, "y": aj.AJ_SWEEP_Y, "auto": aj.AJ_SWEEP_AUTO}[form]
    ctx.set(precision=precision, j_policy=aj.AJ_J_SCALED_DIAG, L=L, maxit=5000, sweep_form=sf)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_EDIVERGED
    # the oracle's first iterate whose residual exceeds 1e8 times that of x^0
    ref = oracle.solve(Q, b, oracle.j_scaled_diag(Q, L), maxit=400, stop=oracle.STOP_NONE, trace=True)
    rel = ref["trace"]["relres"]
    t_div = int(np.nonzero(rel > 1e8 * rel[0])[0][0])
    if form == "y":
        # the explicit-y form reads ||Q y - b|| on every 4th sweep: within a few
        # iterations of the oracle's crossing
        assert t_div - 2 <= info["iters"] <= t_div + 4, (info["iters"], t_div)
    else:
        assert abs(info["iters"] - t_div) <= 1, (info["iters"], t_div)
    # the same context with a valid J solves
    ctx.set(precision=precision, tol=1e-8, maxit=20000)
    _ok_solve(ctx, Q, b)


def test_overflowing_reduction_is_reported_not_faulted():
    Q, b = _poisson(24)
    big = 1e200 * b  # finite entries; ||b||^2 overflows FP64
    assert np.all(np.isfinite(big))
    ctx = aj.from_csr(Q, big)
    ctx.set(maxit=100, format=aj.AJ_FMT_CSR)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_ENONFINITE
    assert info["iters"] == 0
    ctx2 = aj.from_csr(Q, b)
    ctx2.set(tol=1e-8, maxit=20000)
    _ok_solve(ctx2, Q, b)


@pytest.mark.parametrize("fmt", [aj.AJ_FMT_CSR, aj.AJ_FMT_AUTO])
def test_barrier_wait_runs_out(fmt):
    Q, b = _poisson(64)
    ctx = aj.from_csr(Q, b)
    ctx.set(tol=1e-8, maxit=20000, grid_ctas=8, format=fmt)
    aj.inject_barrier_stall(3, 2.0)
    with pytest.raises(aj.AJError) as e:
        ctx.solve()
    assert e.value.status == aj.AJ_ETIMEOUT
    # the hook was one shot: the same context now solves, bit for bit like a fresh one
    x = _ok_solve(ctx, Q, b)
    fresh = aj.from_csr(Q, b)
    fresh.set(tol=1e-8, maxit=20000, grid_ctas=8, format=fmt)
    np.testing.assert_array_equal(x, _ok_solve(fresh, Q, b))
    # a CTA number beyond the grid withholds nothing
    aj.inject_barrier_stall(100000, 2.0)
    np.testing.assert_array_equal(x, _ok_solve(ctx, Q, b))


def test_allocation_failure_in_create_and_set():
    Q, b = _poisson(32)
    # aj_create makes one pool allocation (every array of the context's base)
    aj.inject_alloc_failure(0)
    with pytest.raises(aj.AJError) as e:
        aj.from_csr(Q, b)
    assert e.value.status == aj.AJ_ENOMEM
    aj.inject_alloc_failure(-1)
    ctx = aj.from_csr(Q, b)
    aj.inject_alloc_failure(2)
    with pytest.raises(aj.AJError) as e:
        ctx.set(precision="fp32_ir", tol=1e-8, maxit=20000)
    assert e.value.status == aj.AJ_ENOMEM
    aj.inject_alloc_failure(-1)
    ctx.set(precision="fp32_ir", tol=1e-8, maxit=20000)
    _ok_solve(ctx, Q, b)
    # a context whose aj_set failed solves with the default parameters
    aj.inject_alloc_failure(0)
    with pytest.raises(aj.AJError):
        ctx.set(precision="df64", tol=1e-8, maxit=20000)
    aj.inject_alloc_failure(-1)
    x, info = ctx.solve()
    assert info["status"] == aj.AJ_OK and info["relres"] <= 1e-8
