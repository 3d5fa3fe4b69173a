"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: after a fixed number of iterations the iterates agree to relative
||x_gpu - x_oracle|| <= 1e-10 (FP64 and the double-float policy); every solve
to tolerance reaches an FP64-verified relative residual <= tol.  The oracle
always runs with the GPU's restart schedule forced, and oracle.schedule checks
that schedule against the rule of Algorithm alg-apg-re: the spacing
t > K_re + K_ell exactly, and the decision on d = <Q y - b, x^t - x^{t-1}>
(summed in different orders on the two sides) the oracle's own except at a
rounding-level tie, |d| <= 1e-12 ||Q y - b|| ||x^t - x^{t-1}||.  Three tests
require the oracle's own schedule outright: a solve with six restarts and no
near tie, the strict spacing at K_0 = 64, and ties (d = 0) that restart.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import dense
from oracle import schedule
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402

REL = 1e-10


def _relres(Q, b, x):
    r = b - oracle.spmv(Q, x)
    bn = np.linalg.norm(b)
    return np.linalg.norm(r) / bn if bn > 0 else np.linalg.norm(r)


def _gpu(Q, b, nrhs=1, device=None, **kw):
    ctx = aj.from_csr(Q, b, nrhs=nrhs, device=device)
    ctx.set(**kw)
    x, info = ctx.solve()
    return ctx, x, info


def _oracle_J(Q, j_policy, L=None):
    if j_policy == aj.AJ_J_ABSROWSUM:
        return oracle.j_absrowsum(Q)
    return oracle.j_scaled_diag(Q, L)


FORMS = {"lazy": aj.AJ_SWEEP_LAZY, "stored": aj.AJ_SWEEP_STORED, "delta": aj.AJ_SWEEP_DELTA,
         "y": aj.AJ_SWEEP_Y}


def _compare_fixed(Q, b, T, precision="fp64", restart=True, momentum=True, j_policy=0, L=0.0,
                   x0=None, tol_rel=REL, form="auto"):
    ctx, x, info = _gpu(Q, b, precision=precision, stop=aj.AJ_STOP_NONE, maxit=T,
                        restart=int(restart), momentum=int(momentum), j_policy=j_policy, L=L,
                        x0=x0, sweep_form=FORMS.get(form, aj.AJ_SWEEP_AUTO))
    assert info["iters"] == T and info["status"] == aj.AJ_EMAXIT
    J = _oracle_J(Q, j_policy, L if L else info["L_used"])
    sched = ctx.restart_log()
    assert len(sched) == info["restarts"]
    # the GPU's restart decisions, each the rule's own up to a rounding-level tie
    ref = schedule.replay(Q, b, sched, T, J=J, restart=restart, momentum=momentum, x0=x0,
                          precision="df64" if precision == "df64" else "fp64")
    err = np.linalg.norm(x - ref["x"]) / max(np.linalg.norm(ref["x"]), 1e-300)
    assert err <= tol_rel, (err, sched)
    return ctx, x, info, ref


# ---------------------------------------------------------------- fixed-iteration parity
@pytest.mark.parametrize("form", ["lazy", "stored", "delta", "y"])
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_poisson64_200_iterations_match_oracle(precision, form):
    if form == "delta" and precision != "fp64":
        pytest.skip("the difference form is built for FP64 only")
    Q, b, xs = synth.workload("poisson2d_64")
    _compare_fixed(Q, b, 200, precision=precision, form=form)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_difference_form_equals_stored_form_bitwise(nrhs):
    """x + beta*delta with delta kept from the previous sweep is the same
    rounded operation as x + beta*(x - x_prev): identical iterates."""
    Q = synth.chung_lu_laplacian(5000, seed=81, mean_degree=10.0)  # long rows too
    B = np.stack([synth.rhs(Q, synth.uniform(Q["n"], 60 + r)) for r in range(nrhs)], axis=1)
    bc = np.ascontiguousarray(B.T).reshape(-1)
    out = {}
    for form in ("stored", "delta"):
        ctx = aj.from_csr(Q, bc, nrhs=nrhs)
        ctx.set(tol=1e-10, maxit=20000, sweep_form=FORMS[form], grid_ctas=16)
        x, info = ctx.solve(per_rhs=True)
        out[form] = (x, [i["iters"] for i in info])
    np.testing.assert_array_equal(out["stored"][0], out["delta"][0])
    assert out["stored"][1] == out["delta"][1]


def test_difference_form_is_fp64_only():
    Q, b, xs = synth.workload("poisson2d_64")
    ctx = aj.from_csr(Q, b)
    with pytest.raises(aj.AJError):
        ctx.set(precision="fp32_ir", sweep_form=aj.AJ_SWEEP_DELTA)


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32_ir", "bf16_ir"])
def test_lazy_and_stored_forms_agree(precision):
    # the two sweep forms compute the same iterates up to rounding
    Q, b, xs = synth.workload("poisson2d_40")
    T = 150
    xs_ = {}
    for form in FORMS:
        if form == "delta" and precision != "fp64":
            continue  # built for FP64 only
        ctx, x, info = _gpu(Q, b, precision=precision, stop=aj.AJ_STOP_NONE, maxit=T,
                            sweep_form=FORMS[form], restart=0)
        assert info["iters"] == T
        xs_[form] = x
    tol = 1e-12 if precision in ("fp64", "df64") else 1e-4
    assert np.linalg.norm(xs_["lazy"] - xs_["stored"]) <= tol * np.linalg.norm(xs_["lazy"])
    assert np.linalg.norm(xs_["y"] - xs_["stored"]) <= tol * np.linalg.norm(xs_["lazy"])
    if "delta" in xs_:
        np.testing.assert_array_equal(xs_["delta"], xs_["stored"])


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_no_restart_and_jacobi_modes_match_oracle(precision):
    Q, b, xs = synth.workload("poisson2d_24")
    _compare_fixed(Q, b, 150, precision=precision, restart=False)
    # beta = 0 with J = D: classical Jacobi (eq. jacobi) on a diagonally dominant SPD system
    _compare_fixed(Q, b, 60, precision=precision, restart=False, momentum=False,
                   j_policy=aj.AJ_J_SCALED_DIAG, L=1.0)


@pytest.mark.parametrize("form", ["lazy", "stored", "y"])
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_ragged_tail_and_long_rows(precision, form):
    # n = 300 rows of length 300 (> 32: the warp-cooperative path), n not a multiple of 256
    Q = synth.sdd(300)
    b = np.ones(300)
    _compare_fixed(Q, b, 80, precision=precision, form=form)
    # a 3-D grid with a ragged last tile and boundary rows of every length
    Q, b, xs = synth.workload("poisson3d_13")
    assert Q["n"] % 256 != 0
    _compare_fixed(Q, b, 120, precision=precision, form=form)


def test_singular_laplacian_with_empty_rows():
    n = 2000
    Q = synth.chung_lu_laplacian(n, seed=11, mean_degree=4.0)
    assert (np.diff(Q["row_ptr"]) == 0).any()
    xs = synth.uniform(n, 12)
    b = synth.rhs(Q, xs)
    ctx, x, info, ref = _compare_fixed(Q, b, 150)
    empty = np.diff(Q["row_ptr"]) == 0
    assert np.all(x[empty] == 0.0)


def test_scaled_diag_given_L_and_estimated_L():
    N = 40
    Q, b, xs = synth.workload("poisson2d_%d" % N)
    Lt = 1.0 + math.cos(math.pi / (N + 1))
    _compare_fixed(Q, b, 100, j_policy=aj.AJ_J_SCALED_DIAG, L=Lt)
    ctx, x, info = _gpu(Q, b, j_policy=aj.AJ_J_SCALED_DIAG, L=0.0, maxit=5000)
    # power iteration with a 2 % margin, capped by the Gershgorin bound 2
    assert Lt * (1 - 1e-6) <= info["L_used"] <= min(2.0, Lt * 1.03)
    assert info["status"] == aj.AJ_OK and info["relres"] <= 1e-8


def test_x0_and_device_pointers():
    Q, b, xs = synth.workload("poisson2d_32")
    x0 = synth.uniform(Q["n"], 5)
    _compare_fixed(Q, b, 90, x0=x0)
    ctx = aj.from_csr(Q, b, device="cuda")
    x0d = torch.from_numpy(x0).cuda()
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=90, x0=x0d)
    out = torch.empty(Q["n"], dtype=torch.float64, device="cuda")
    _, info = ctx.solve(out=out)
    ref = schedule.replay(Q, b, ctx.restart_log(), 90, J=oracle.j_absrowsum(Q), x0=x0)
    xg = out.cpu().numpy()
    assert np.linalg.norm(xg - ref["x"]) <= REL * np.linalg.norm(ref["x"])


# ---------------------------------------------------------------- solves to tolerance
@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32_ir", "bf16_ir"])
def test_poisson64_solve_to_1e8(precision):
    Q, b, xs = synth.workload("poisson2d_64")
    ctx, x, info = _gpu(Q, b, precision=precision, tol=1e-8, maxit=20000)
    assert info["status"] == aj.AJ_OK
    rr = _relres(Q, b, x)
    assert rr <= 1e-8 and abs(rr - info["relres"]) <= 1e-3 * rr + 1e-15
    ref = oracle.solve(Q, b, oracle.j_absrowsum(Q), tol=1e-8, maxit=20000)
    if precision in ("fp64", "df64"):
        # same stop rule on the same iterates: same iteration count up to a flipped decision
        assert abs(info["iters"] - ref["iters"]) <= max(3, 0.02 * ref["iters"])
    # error against the oracle's converged solution in the Q-norm
    A = dense.to_dense(Q)
    e = x - ref["x"]
    assert math.sqrt(e @ (A @ e)) <= 1e-6 * math.sqrt(ref["x"] @ (A @ ref["x"]))


def test_objective_gap_stop_matches_oracle():
    n = 400
    Q = synth.sdd(n)
    b = np.ones(n)
    fstar = -n / 2.0
    ctx, x, info = _gpu(Q, b, stop=aj.AJ_STOP_OBJGAP, tol=1e-10, fstar=fstar, maxit=5000)
    ref = oracle.solve(Q, b, oracle.j_absrowsum(Q), stop=oracle.STOP_OBJGAP, tol=1e-10,
                       fstar=fstar, maxit=5000)
    assert info["status"] == aj.AJ_OK and ref["converged"]
    assert abs(info["iters"] - ref["iters"]) <= 2
    assert info["objgap"] <= 1e-10
    np.testing.assert_allclose(x, np.ones(n), atol=1e-4)


def test_zero_rhs_and_tiny_systems():
    Q = synth.poisson2d(8)
    ctx, x, info = _gpu(Q, np.zeros(64))
    assert info["iters"] == 0 and info["status"] == aj.AJ_OK and np.all(x == 0)
    # n = 1
    Q1 = {"n": 1, "row_ptr": np.array([0, 1], np.int32), "col": np.array([0], np.int32),
          "val": np.array([3.0])}
    ctx, x, info = _gpu(Q1, np.array([6.0]))
    assert info["status"] == aj.AJ_OK and abs(x[0] - 2.0) <= 1e-12


# ---------------------------------------------------------------- several right-hand sides
@pytest.mark.parametrize("form", ["auto", "y"])
@pytest.mark.parametrize("nrhs", [2, 3, 4])
@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32_ir"])
def test_multi_rhs_equals_single(nrhs, precision, form):
    Q = synth.poisson2d(30)
    n = Q["n"]
    B = np.stack([synth.rhs(Q, synth.uniform(n, 20 + r)) for r in range(nrhs)], axis=1)
    bc = np.ascontiguousarray(B.T).reshape(-1)  # column-major n x nrhs
    ctx = aj.from_csr(Q, bc, nrhs=nrhs)
    # the same sweep form for both runs (AUTO gives FP64, and FP32 values in
    # the stencil format, with one right-hand side the explicit-y form, with
    # several the difference or lazy form), and the same grid, so the FP64
    # reductions are summed in the same order
    sf = aj.AJ_SWEEP_Y if form == "y" else (aj.AJ_SWEEP_DELTA if precision == "fp64" else aj.AJ_SWEEP_LAZY)
    ctx.set(precision=precision, tol=1e-9, maxit=10000, grid_ctas=8, sweep_form=sf)
    X, infos = ctx.solve(per_rhs=True)
    X = X.reshape(nrhs, n)
    for r in range(nrhs):
        c1, x1, i1 = _gpu(Q, B[:, r], precision=precision, tol=1e-9, maxit=10000, grid_ctas=8,
                          sweep_form=sf)
        assert infos[r]["iters"] == i1["iters"]
        np.testing.assert_array_equal(X[r], x1)
        assert _relres(Q, B[:, r], X[r]) <= 1e-9


@pytest.mark.parametrize("nrhs", [2, 3, 4])
@pytest.mark.parametrize("case", ["poisson_lazy", "poisson_stored", "poisson_y", "long_rows", "sell_powerlaw",
                                  "sell_powerlaw_y"])
def test_multi_rhs_200_iterations_match_oracle(nrhs, case):
    """Several right-hand sides share a row's lanes (lane r gathers column r
    of the interleaved vectors); every column must follow the FP64 oracle."""
    if case.startswith("poisson"):
        Q = synth.poisson2d(41)  # n = 1681: a ragged last tile for every lane count
        kw = dict(sweep_form=FORMS[case.split("_")[1]])
    elif case == "long_rows":
        # power-law rows: the hubs exceed the warp-cooperative threshold of 32 entries
        Q = synth.chung_lu_laplacian(3000, seed=19, mean_degree=12.0)
        kw = dict(format=aj.AJ_FMT_CSR)
    else:
        Q = synth.chung_lu_laplacian(20000, seed=29)
        kw = dict(format=aj.AJ_FMT_SELL, sell_sigma=256, sell_lmax=16)
        if case.endswith("_y"):
            kw["sweep_form"] = aj.AJ_SWEEP_Y
    n = Q["n"]
    B = np.stack([synth.rhs(Q, synth.uniform(n, 40 + r)) for r in range(nrhs)], axis=1)
    ctx = aj.from_csr(Q, np.ascontiguousarray(B.T).reshape(-1), nrhs=nrhs)
    T = 200
    ctx.set(stop=aj.AJ_STOP_NONE, maxit=T, **kw)
    X, infos = ctx.solve(per_rhs=True)
    X = X.reshape(nrhs, n)
    J = oracle.j_absrowsum(Q)
    for r in range(nrhs):
        assert infos[r]["iters"] == T
        ref = schedule.replay(Q, B[:, r], ctx.restart_log(r), T, J=J)
        err = np.linalg.norm(X[r] - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= REL, (r, err)
    if case == "long_rows":
        assert np.diff(Q["row_ptr"]).max() > 32


# ---------------------------------------------------------------- checkpoint / resume
@pytest.mark.parametrize("form", ["lazy", "stored", "delta", "y"])
def test_resume_is_bit_identical(form):
    Q, b, xs = synth.workload("poisson2d_48")
    full = aj.from_csr(Q, b)
    full.set(stop=aj.AJ_STOP_NONE, maxit=400, sweep_form=FORMS[form])
    xf, inf_f = full.solve()
    part = aj.from_csr(Q, b)
    part.set(stop=aj.AJ_STOP_NONE, maxit=170, sweep_form=FORMS[form])
    part.solve()
    blob = part.get_state()
    other = aj.from_csr(Q, b)
    other.set(stop=aj.AJ_STOP_NONE, maxit=400, sweep_form=FORMS[form])
    other.set_state(blob)
    xr, inf_r = other.solve()
    np.testing.assert_array_equal(xr, xf)
    assert inf_r["restarts"] == inf_f["restarts"]


# ---------------------------------------------------------------- invalid input
def test_invalid_matrices_rejected():
    good = synth.poisson2d(6)
    bad = dict(good, row_ptr=good["row_ptr"].copy())
    bad["row_ptr"][3] = bad["row_ptr"][2] - 1
    with pytest.raises(aj.AJError) as e:
        aj.from_csr(bad, np.ones(36))
    assert e.value.status == aj.AJ_EINVAL
    bad = dict(good, col=good["col"].copy())
    bad["col"][5] = 36
    with pytest.raises(aj.AJError):
        aj.from_csr(bad, np.ones(36))
    bad = dict(good, val=good["val"].copy())
    bad["val"][0] = -4.0
    with pytest.raises(aj.AJError):
        aj.from_csr(bad, np.ones(36))
    # a non-finite right-hand side, in the first or a later column
    for k, v in ((3, np.nan), (35, np.inf), (36 + 7, -np.inf)):
        bb = np.ones(72)
        bb[k] = v
        with pytest.raises(aj.AJError) as e:
            aj.from_csr(good, bb, nrhs=2)
        assert e.value.status == aj.AJ_EINVAL
    ctx = aj.from_csr(good, np.ones(36))
    with pytest.raises(aj.AJError):
        ctx.set(K0=1)


# ---------------------------------------------------------------- the restart rule itself
def _stop_is_clear(tr_relres, iters, tol):
    # the residual near tol carries a relative rounding error of about eps / tol
    # on either side; the stop iteration is fixed when it is clear of that
    return all(abs(tr_relres[t] / tol - 1.0) > 1e-2 for t in (iters - 1, iters))


@pytest.mark.parametrize("precision,form", [("fp64", "auto"), ("fp64", "lazy"), ("fp64", "stored"),
                                            ("fp64", "delta"), ("fp64", "y"), ("df64", "auto"),
                                            ("df64", "y")])
@pytest.mark.parametrize("fmt", ["csr", "auto"])
def test_restart_schedule_equals_the_oracles(precision, form, fmt):
    """2-D Poisson 64 x 64 to relative residual 1e-12: six restarts, and every
    d_t is at least 1e-4 of its scale ||g|| ||x^t - x^{t-1}||, so no decision is
    near a tie.  The GPU must take exactly the oracle's restart iterations
    (Algorithm alg-apg-re) and stop at the oracle's iteration."""
    Q, b, _ = synth.workload("poisson2d_64")
    J = oracle.j_absrowsum(Q)
    tol = 1e-12
    ref = oracle.solve(Q, b, J, tol=tol, maxit=20000, trace=True)
    nat = [int(t) for t in np.nonzero(ref["trace"]["restart"])[0]]
    assert len(nat) >= 3
    F = aj.AJ_FMT_CSR if fmt == "csr" else aj.AJ_FMT_AUTO
    ctx, x, info = _gpu(Q, b, precision=precision, tol=tol, maxit=20000, format=F,
                        sweep_form=FORMS.get(form, aj.AJ_SWEEP_AUTO))
    assert ctx.restart_log() == nat
    assert info["restarts"] == len(nat)
    if _stop_is_clear(ref["trace"]["relres"], ref["iters"], tol):
        assert info["iters"] == ref["iters"]
    else:
        assert abs(info["iters"] - ref["iters"]) <= 1


def test_restart_spacing_is_strict():
    """K_0 = 64 on 2-D Poisson 32 x 32: the oracle's d is already >= 0 (at 6 %
    of its scale) at t = 64 = K_re + K_0, so the strict t > K_re + K_ell
    restarts at 65, where t >= K_re + K_ell would restart at 64."""
    Q, b, _ = synth.workload("poisson2d_32")
    J = oracle.j_absrowsum(Q)
    nat, _ = schedule.natural(Q, b, 200, J=J, K0=64)
    assert nat == [65, 200]
    for F in (aj.AJ_FMT_CSR, aj.AJ_FMT_AUTO):
        ctx, x, info = _gpu(Q, b, stop=aj.AJ_STOP_NONE, maxit=200, K0=64, format=F)
        assert ctx.restart_log() == nat


def test_tie_restarts():
    """b = 0 from x^0 = 0: g = 0 and x^t - x^{t-1} = 0 exactly, so d = 0, and
    the non-strict d >= 0 restarts as soon as the spacing allows: t = 3, 8,
    17, 34 for K_0 = 2."""
    Q = synth.poisson2d(8)
    z = np.zeros(Q["n"])
    nat, _ = schedule.natural(Q, z, 40, J=oracle.j_absrowsum(Q))
    assert nat == [3, 8, 17, 34]
    for form in FORMS.values():
        ctx, x, info = _gpu(Q, z, stop=aj.AJ_STOP_NONE, maxit=40, sweep_form=form)
        assert ctx.restart_log() == nat and np.all(x == 0.0)
