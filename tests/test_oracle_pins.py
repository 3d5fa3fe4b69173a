"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formula: each checks it against a
closed form, a library routine on a different formulation, an identity from
the paper's analysis, or brute force on a tiny input.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = line.split("=", 1)
            vals[k.strip()] = v.strip()
    return vals


def _random_csr(n, density, seed, symmetric=False, spd_shift=0.0):
    rng = np.random.default_rng(seed)
    A = np.where(rng.random((n, n)) < density, rng.uniform(-1, 1, (n, n)), 0.0)
    if symmetric:
        A = np.triu(A, 1)
        A = A + A.T
        A += np.diag(np.abs(A).sum(1) + spd_shift)
    return _dense_to_csr(A), A


def _dense_to_csr(A):
    n = A.shape[0]
    rp = [0]
    ci, v = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        ci.extend(nz.tolist())
        v.extend(A[i, nz].tolist())
        rp.append(len(ci))
    return {"n": n, "row_ptr": np.array(rp, np.int32), "col": np.array(ci, np.int32),
            "val": np.array(v, np.float64)}


# --------------------------------------------------------------------------- SpMV
def test_spmv_matches_dense_nonsymmetric():
    # a non-symmetric matrix so a transposed operand would be caught
    Q, A = _random_csr(37, 0.2, 11)
    y = np.random.default_rng(1).standard_normal(37)
    np.testing.assert_allclose(oracle.spmv(Q, y), A @ y, rtol=1e-13, atol=1e-13)


def test_spmv_empty_rows_and_empty_matrix():
    Q = {"n": 4, "row_ptr": np.array([0, 0, 2, 2, 3], np.int32),
         "col": np.array([0, 3, 1], np.int32), "val": np.array([2.0, -1.0, 5.0])}
    y = np.array([1.0, 2.0, 3.0, 4.0])
    np.testing.assert_array_equal(oracle.spmv(Q, y), [0.0, 2.0 - 4.0, 0.0, 10.0])
    Z = {"n": 0, "row_ptr": np.zeros(1, np.int32), "col": np.zeros(0, np.int32),
         "val": np.zeros(0)}
    assert oracle.spmv(Z, np.zeros(0)).shape == (0,)


def test_sdd_matrix_times_ones_is_ones():
    g = _read_golden("sdd_section4_1.txt")
    assert g["diag_value"] == "n" and g["offdiag_value"] == "-1"
    Q = synth.sdd(300)
    np.testing.assert_array_equal(oracle.spmv(Q, np.ones(300)), np.ones(300))


# --------------------------------------------------------------------------- J
def test_j_absrowsum_poisson_hand_values():
    N = 5
    J = oracle.j_absrowsum(synth.poisson2d(N)).reshape(N, N)
    assert J[2, 2] == 8.0      # interior: 4 + 4 neighbours
    assert J[0, 2] == 7.0      # edge: 4 + 3
    assert J[0, 0] == 6.0      # corner: 4 + 2
    J3 = oracle.j_absrowsum(synth.poisson3d(4)).reshape(4, 4, 4)
    assert J3[1, 1, 1] == 12.0 and J3[0, 0, 0] == 9.0


def test_j_absrowsum_sdd_is_2n_minus_1():
    n = 200
    np.testing.assert_array_equal(oracle.j_absrowsum(synth.sdd(n)), np.full(n, 2.0 * n - 1.0))


def test_j_zero_row_gets_one():
    Q = synth.from_edges(5, [0, 1], [1, 2], [1.0, 2.0])  # vertices 3, 4 isolated
    J = oracle.j_absrowsum(Q)
    assert J[3] == 1.0 and J[4] == 1.0
    assert J[1] == 3.0 + 3.0
    Js = oracle.j_scaled_diag(Q, 2.0)
    assert Js[3] == 1.0 and Js[1] == 6.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_S_is_psd_for_absrowsum(seed):
    # eq. J-diag makes S = J - Q positive semidefinite (Gershgorin), Section 3
    Q, A = _random_csr(40, 0.15, seed, symmetric=True)
    J = oracle.j_absrowsum(Q)
    w = np.linalg.eigvalsh(np.diag(J) - A)
    assert w.min() >= -1e-12 * abs(w).max()


def test_poisson_step_constant_closed_form():
    for N in (6, 8, 11):
        L = dense.step_constant_L(synth.poisson2d(N))
        assert abs(L - (1.0 + math.cos(math.pi / (N + 1)))) < 1e-12
    for N in (4, 5):
        L = dense.step_constant_L(synth.poisson3d(N))
        assert abs(L - (1.0 + math.cos(math.pi / (N + 1)))) < 1e-12


def test_scaled_diag_with_L_gives_psd_S():
    Q = synth.poisson2d(7)
    L = dense.step_constant_L(Q)
    J = oracle.j_scaled_diag(Q, L)
    w = np.linalg.eigvalsh(np.diag(J) - dense.to_dense(Q))
    assert w.min() >= -1e-12


# --------------------------------------------------------------------------- fixed point
def test_converges_to_direct_solution_spd():
    Q, A = _random_csr(60, 0.1, 5, symmetric=True, spd_shift=0.5)
    xs = np.random.default_rng(2).uniform(-1, 1, 60)
    b = A @ xs
    r = oracle.solve(Q, b, oracle.j_absrowsum(Q), maxit=20000, tol=1e-14)
    assert r["converged"]
    np.testing.assert_allclose(r["x"], np.linalg.solve(A, b), rtol=0, atol=1e-11)


def test_sdd_reaches_all_ones():
    # Section 4.1: x* = 1; objective-gap stop at 1e-10 as in the paper, then tighter
    n = 1000
    Q = synth.sdd(n)
    b = np.ones(n)
    fstar = -n / 2.0
    r = oracle.solve(Q, b, oracle.j_absrowsum(Q), maxit=5000, stop=oracle.STOP_OBJGAP,
                     tol=1e-10, fstar=fstar)
    assert r["converged"] and r["iters"] < 5000
    r2 = oracle.solve(Q, b, oracle.j_absrowsum(Q), maxit=20000, tol=1e-13)
    np.testing.assert_allclose(r2["x"], np.ones(n), rtol=0, atol=1e-10)


def test_sdd_acceleration_beats_jacobi_within_5000():
    # Section 4.1: (weighted) Jacobi do not reach the tolerance in 5000 iterations on
    # these systems, while the accelerated methods do.
    n = 1000
    Q = synth.sdd(n)
    b = np.ones(n)
    fstar = -n / 2.0
    kw = dict(maxit=5000, stop=oracle.STOP_OBJGAP, tol=1e-10, fstar=fstar)
    jac = oracle.solve(Q, b, oracle.j_scaled_diag(Q, 1.0), restart=False, momentum=False, **kw)
    aj = oracle.solve(Q, b, oracle.j_absrowsum(Q), restart=False, **kw)
    ajr = oracle.solve(Q, b, oracle.j_absrowsum(Q), restart=True, **kw)
    assert not jac["converged"]
    assert aj["converged"] and ajr["converged"]
    assert ajr["iters"] <= aj["iters"]


# --------------------------------------------------------------------------- Jacobi special cases
def test_beta_zero_J_eq_D_is_classical_jacobi_splitting_form():
    # eq. jacobi, splitting form x+ = D^-1 (b - (L + L^T) x), computed densely
    Q, A = _random_csr(30, 0.2, 9, symmetric=True, spd_shift=1.0)
    b = np.random.default_rng(3).standard_normal(30)
    D = np.diag(A)
    x = np.zeros(30)
    for _ in range(25):
        x = (b - (A - np.diag(D)) @ x) / D
    r = oracle.solve(Q, b, oracle.j_scaled_diag(Q, 1.0), restart=False, momentum=False,
                     maxit=25, stop=oracle.STOP_NONE)
    np.testing.assert_allclose(r["x"], x, rtol=1e-12, atol=1e-13)


def test_jacobi_contraction_on_poisson_is_cos_pi_over_n_plus_1():
    N = 9
    Q = synth.poisson2d(N)
    s = np.sin(np.arange(1, N + 1) * math.pi / (N + 1))
    v = np.outer(s, s).reshape(-1)  # slowest mode
    rho = math.cos(math.pi / (N + 1))
    r = oracle.solve(Q, np.zeros(N * N), oracle.j_scaled_diag(Q, 1.0), restart=False,
                     momentum=False, maxit=7, stop=oracle.STOP_NONE, x0=v)
    np.testing.assert_allclose(r["x"], rho ** 7 * v, rtol=1e-12, atol=1e-14)


def test_weighted_jacobi_optimal_rate_on_sdd():
    # eq. weighted-jacobi with omega_opt = 2/(lmin + lmax) of D^-1 Q; for the SDD matrix
    # D^-1 Q has eigenvalues (n+1)/n and 1/n, so omega_opt = 2n/(n+2), rate n/(n+2).
    n = 50
    Q = synth.sdd(n)
    A = dense.to_dense(Q)
    w = np.linalg.eigvalsh(A / n)
    omega = 2.0 / (w[0] + w[-1])
    assert abs(omega - 2.0 * n / (n + 2)) < 1e-12
    # start from an eigenvector of the (n+1) eigenvalue: error contracts by exactly n/(n+2)
    e = np.zeros(n)
    e[0], e[1] = 1.0, -1.0
    r = oracle.solve(Q, np.zeros(n), oracle.j_scaled_diag(Q, 1.0 / omega), restart=False,
                     momentum=False, maxit=3, stop=oracle.STOP_NONE, x0=e)
    np.testing.assert_allclose(r["x"], (-(n / (n + 2.0))) ** 3 * e, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------- analysis identities
def _tiny_spd():
    Q, A = _random_csr(24, 0.25, 21, symmetric=True, spd_shift=0.05)
    xs = np.random.default_rng(4).uniform(-1, 1, 24)
    return Q, A, xs, A @ xs


def _tiny_laplacian():
    rng = np.random.default_rng(8)
    n = 20
    u, v, w = [], [], []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < 0.25 or j == i + 1:
                u.append(i); v.append(j); w.append(rng.uniform(0.5, 1.5))
    Q = synth.from_edges(n, u, v, w)
    A = dense.to_dense(Q)
    xs = rng.uniform(-1, 1, n)
    return Q, A, xs, A @ xs


@pytest.mark.parametrize("case", [_tiny_spd, _tiny_laplacian])
def test_prox_optimality_every_iterate(case):
    # Lemma lemma-diff-f proof: Q x^t - b + S (x^t - y^t) = 0 with S = J - Q
    Q, A, xs, b = case()
    J = oracle.j_absrowsum(Q)
    T = 60
    r = oracle.solve(Q, b, J, restart=False, maxit=T, stop=oracle.STOP_NONE, trace_iterates=True)
    X, Y = r["trace"]["x"], r["trace"]["y"]
    S = np.diag(J) - A
    for t in range(1, T + 1):
        res = A @ X[t] - b + S @ (X[t] - Y[t])
        assert np.abs(res).max() <= 1e-12 * (1 + np.abs(b).max())


def test_alpha_sequence_facts():
    Q, A, xs, b = _tiny_spd()
    r = oracle.solve(Q, b, oracle.j_absrowsum(Q), restart=False, maxit=300,
                     stop=oracle.STOP_NONE, trace=True)
    a = r["trace"]["alpha"]
    assert a[1] == 1.0
    for t in range(1, 301):
        assert a[t] >= (t + 1) / 2.0 - 1e-12           # Theorem thm-convergence proof
    for t in range(2, 301):                              # identity used in Lemma lemma-recursive
        assert abs(a[t - 1] ** 2 - a[t] * (a[t] - 1.0)) <= 1e-12 * a[t] ** 2
    beta = r["trace"]["beta"]
    for t in range(1, 300):
        assert abs(beta[t] - (a[t] - 1.0) / a[t + 1]) <= 1e-15
        assert 0.0 <= beta[t] < 1.0


@pytest.mark.parametrize("case", [_tiny_spd, _tiny_laplacian])
def test_objective_rate_bound(case):
    # Theorem thm-convergence: 0 <= f(x^t) - f* <= 2 ||x^0 - x*||_S^2 / (t+1)^2
    Q, A, xs, b = case()
    J = oracle.j_absrowsum(Q)
    S = np.diag(J) - A
    fstar = dense.f_value(A, b, xs)
    R2 = xs @ (S @ xs)  # x^0 = 0
    T = 500
    r = oracle.solve(Q, b, J, restart=False, maxit=T, stop=oracle.STOP_NONE, trace=True)
    f = r["trace"]["f"]
    for t in range(1, T + 1):
        gap = f[t] - fstar
        assert gap >= -1e-12
        assert gap <= 2.0 * R2 / (t + 1) ** 2 + 1e-12


@pytest.mark.parametrize("case", [_tiny_spd, _tiny_laplacian])
def test_energy_nonincreasing(case):
    # Lemma lemma-recursive: alpha_t^2 (f(x^t) - f*) + 1/2 <w^t, S w^t> is non-increasing,
    # w^t = alpha_t x^t - (alpha_t - 1) x^{t-1} - x*
    Q, A, xs, b = case()
    J = oracle.j_absrowsum(Q)
    S = np.diag(J) - A
    fstar = dense.f_value(A, b, xs)
    T = 200
    r = oracle.solve(Q, b, J, restart=False, maxit=T, stop=oracle.STOP_NONE, trace_iterates=True)
    X = r["trace"]["x"]
    a = r["trace"]["alpha"]
    E = []
    for t in range(1, T + 1):
        w = a[t] * X[t] - (a[t] - 1.0) * X[t - 1] - xs
        E.append(a[t] ** 2 * (dense.f_value(A, b, X[t]) - fstar) + 0.5 * w @ (S @ w))
    E0 = 0.5 * xs @ (S @ xs)  # alpha_0 = 0, w^0 = -x* with x^0 = 0
    assert E[0] <= E0 + 1e-12
    # rounding of f(x^t) - f* is amplified by alpha_t^2 (about t^2 / 4)
    for t in range(1, T):
        slack = 1e-13 * a[t + 1] ** 2 * (1.0 + abs(fstar)) + 1e-12 * E0
        assert E[t] <= E[t - 1] + slack


def test_restart_rules_and_monotone_epochs():
    # Algorithm alg-apg-re and Lemma lemma-re-descend / Theorem thm-convergence-re
    Q = synth.poisson2d(24)
    xs = synth.uniform(Q["n"], 7)
    b = synth.rhs(Q, xs)
    A = dense.to_dense(Q)
    K0 = 2
    r = oracle.solve(Q, b, oracle.j_absrowsum(Q), restart=True, K0=K0, maxit=1500, tol=1e-12,
                     trace=True)
    tr = r["trace"]
    T = r["iters"]
    rs = [t for t in range(1, T + 1) if tr["restart"][t]]
    assert len(rs) >= 2 and len(rs) == r["restarts"]
    # restarts happen only when <Q y^t - b, x^t - x^{t-1}> >= 0 and spacing exceeds K_ell
    Kre, K = 0, K0
    for t in range(1, T + 1):
        allowed = t > Kre + K
        if tr["restart"][t]:
            assert allowed and tr["d"][t] >= 0.0
            Kre, K = t, 2 * K
        else:
            assert not (allowed and tr["d"][t] >= 0.0)
    # restart count bound  ell <= log2(t + 2) - 1
    ell = 0
    for t in range(1, T + 1):
        ell += int(tr["restart"][t])
        assert ell <= math.log2(t + 2) - 1 + 1e-12
    # objective never rises above the epoch's starting value; epoch starts decrease
    f = tr["f"]
    starts = [0] + rs
    for k, s in enumerate(starts):
        end = starts[k + 1] if k + 1 < len(starts) else T
        for t in range(s, end + 1):
            assert f[t] <= f[s] + 1e-10 * abs(f[s])
    fs = [f[s] for s in starts]
    assert all(fs[i + 1] <= fs[i] + 1e-10 * abs(fs[i]) for i in range(len(fs) - 1))
    assert r["relres"] <= 1e-12


def test_no_restart_mode_is_alg_apg_and_forced_replay_is_exact():
    Q = synth.poisson2d(16)
    b = synth.rhs(Q, synth.uniform(Q["n"], 3))
    J = oracle.j_absrowsum(Q)
    a = oracle.solve(Q, b, J, restart=False, maxit=300, stop=oracle.STOP_NONE, trace=True)
    assert a["restarts"] == 0 and not a["trace"]["restart"].any()
    nat = oracle.solve(Q, b, J, restart=True, maxit=300, stop=oracle.STOP_NONE, trace=True)
    sched = [t for t in range(1, 301) if nat["trace"]["restart"][t]]
    rep = oracle.solve(Q, b, J, restart=True, maxit=300, stop=oracle.STOP_NONE, forced=sched)
    np.testing.assert_array_equal(rep["x"], nat["x"])
    assert rep["restarts"] == nat["restarts"]


# --------------------------------------------------------------------------- singular Laplacians
def test_chung_lu_laplacian_range_and_solution():
    n = 3000
    Q = synth.chung_lu_laplacian(n, seed=5)
    xs = synth.uniform(n, 6)
    b = synth.rhs(Q, xs)
    A = dense.to_dense(Q)
    # symmetric, zero row sums (Laplacian), b in range(Q): sums over each component vanish
    np.testing.assert_array_equal(A, A.T)
    assert np.abs(A.sum(1)).max() < 1e-12
    import scipy.sparse.csgraph as csg
    import scipy.sparse as sp
    ncomp, lab = csg.connected_components(sp.csr_matrix(np.abs(A) > 0), directed=False)
    for c in range(ncomp):
        m = lab == c
        assert abs(b[m].sum()) <= 1e-12 * (1 + np.abs(b).sum())
    J = oracle.j_absrowsum(Q)
    r = oracle.solve(Q, b, J, maxit=20000, tol=1e-10)
    assert r["converged"] and r["relres"] <= 1e-10
    # solutions differ from x* only by null-space components: compare in the Q-seminorm
    e = r["x"] - xs
    assert e @ (A @ e) <= 1e-14 * (xs @ (A @ xs))
    # isolated vertices (empty rows) keep x^0 = 0
    empty = np.diff(Q["row_ptr"]) == 0
    assert np.all(r["x"][empty] == 0.0)
    assert np.isfinite(r["x"]).all() and np.abs(r["x"]).max() < 1e3


def test_relres_stop_semantics_and_zero_rhs():
    Q = synth.poisson2d(8)
    r = oracle.solve(Q, np.zeros(64), oracle.j_absrowsum(Q), tol=1e-8)
    assert r["iters"] == 0 and r["converged"] and np.all(r["x"] == 0)
    b = synth.rhs(Q, synth.uniform(64, 1))
    r = oracle.solve(Q, b, oracle.j_absrowsum(Q), tol=1e-8, maxit=10000, trace=True)
    rr = r["trace"]["relres"]
    t = r["iters"]
    assert rr[t] <= 1e-8 and np.all(rr[:t] > 1e-8)
    np.testing.assert_allclose(np.linalg.norm(b - dense.to_dense(Q) @ r["x"]) / np.linalg.norm(b),
                               r["relres"], rtol=1e-6)


def test_isolated_vertices_keep_initial_value():
    # zero rows: J_kk = 1 and b_k = 0, so x_k stays at x^0_k
    Q = synth.from_edges(6, [0, 1, 3], [1, 2, 4], [1.0, 0.7, 1.2])  # vertex 5 isolated
    xs = np.array([0.3, -0.2, 0.9, 0.1, -0.4, 0.0])
    b = synth.rhs(Q, xs)
    x0 = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.25])
    r = oracle.solve(Q, b, oracle.j_absrowsum(Q), maxit=5000, tol=1e-12, x0=x0)
    assert r["converged"] and r["x"][5] == 0.25


def test_restart_is_a_fresh_start_from_previous_iterate():
    # Section 2.2: a restart at t sets x^t = x^{t-1}, y^{t+1} = x^{t-1}, alpha_{t+1} = 1, so the
    # run continues exactly like Algorithm alg-apg started afresh at x^0 := x^{t-1}.
    Q = synth.poisson2d(12)
    b = synth.rhs(Q, synth.uniform(Q["n"], 9))
    J = oracle.j_absrowsum(Q)
    T, tr = 40, 9
    forced = oracle.solve(Q, b, J, restart=True, maxit=T, stop=oracle.STOP_NONE, forced=[tr],
                          trace_iterates=True)
    head = oracle.solve(Q, b, J, restart=False, maxit=tr - 1, stop=oracle.STOP_NONE)
    fresh = oracle.solve(Q, b, J, restart=False, maxit=T - tr, stop=oracle.STOP_NONE,
                         x0=head["x"], trace_iterates=True)
    X = forced["trace"]["x"]
    np.testing.assert_array_equal(X[tr], X[tr - 1])          # x^t = x^{t-1}
    assert forced["trace"]["f"][tr] == forced["trace"]["f"][tr - 1]
    for s in range(0, T - tr + 1):
        np.testing.assert_array_equal(X[tr + s], fresh["trace"]["x"][s])
    np.testing.assert_array_equal(forced["x"], fresh["x"])


# --------------------------------------------------------------------------- block-diagonal J (eq. J-blkdiag)
def _block_dense(Jb, n):
    s, bs, _ = Jb.shape
    J = np.zeros((s * bs, s * bs))
    for i in range(s):
        J[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs] = Jb[i]
    return J[:n, :n]


def test_j_blkdiag_hand_values_use_the_spectral_norm():
    # Laplacian of the unit-weight graph 0-2, 0-3, 1-2, 2-3; blocks {0, 1}, {2, 3}.
    # Q^{12} = [[-1, -1], [-1, 0]]: (Q^{12})^T Q^{12} = [[2, 1], [1, 1]] has eigenvalues
    # (3 +- sqrt 5) / 2, so ||Q^{12}||_2 = sqrt((3 + sqrt 5) / 2) = phi, the golden ratio
    # (the Frobenius norm sqrt 3, the largest entry 1 and the row-sum norm 2 all differ).
    Q = synth.from_edges(4, [0, 0, 1, 2], [2, 3, 2, 3], [1.0, 1.0, 1.0, 1.0])
    phi = (1 + math.sqrt(5)) / 2
    Jb = oracle.j_blkdiag(Q, 2)
    np.testing.assert_allclose(Jb[0], [[2 + phi, 0], [0, 1 + phi]], rtol=1e-15)
    np.testing.assert_allclose(Jb[1], [[3 + phi, -1], [-1, 2 + phi]], rtol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_j_blkdiag_of_size_one_is_j_diag(seed):
    # 1 x 1 blocks: ||Q_ij||_2 = |Q_ij|, so eq. J-blkdiag reduces to eq. J-diag
    Q, _ = _random_csr(30, 0.3, 40 + seed, symmetric=True, spd_shift=0.1)
    for M in (Q, synth.chung_lu_laplacian(300, seed=seed + 2, mean_degree=5.0)):
        np.testing.assert_allclose(oracle.j_blkdiag(M, 1)[:, 0, 0], oracle.j_absrowsum(M), rtol=1e-15)


@pytest.mark.parametrize("bs", [2, 3, 5, 8])
@pytest.mark.parametrize("case", [_tiny_spd, _tiny_laplacian])
def test_j_blkdiag_gives_psd_S_and_pd_J(case, bs):
    # Section 3: S = J - Q is positive semidefinite and J positive definite
    Q, A, _, _ = case()
    J = _block_dense(oracle.j_blkdiag(Q, bs), Q["n"])
    np.testing.assert_array_equal(J, J.T)
    scale = np.abs(A).max()
    assert np.linalg.eigvalsh(J - A)[0] >= -1e-12 * scale
    assert np.linalg.eigvalsh(J)[0] > 1e-9 * scale


def test_one_block_is_q_and_solves_in_one_step():
    # s = 1: J = Q, so x^1 = y^1 - Q^{-1}(Q y^1 - b) = Q^{-1} b
    Q, A, xs, b = _tiny_spd()
    Jb = oracle.j_blkdiag(Q, 32)
    np.testing.assert_allclose(_block_dense(Jb, Q["n"]), A, rtol=0, atol=0)
    r = oracle.solve(Q, b, Jblk=Jb, maxit=1, stop=oracle.STOP_NONE)
    np.testing.assert_allclose(r["x"], xs, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("bs", [3, 4])
@pytest.mark.parametrize("case", [_tiny_spd, _tiny_laplacian])
def test_block_update_prox_optimality_every_iterate(case, bs):
    # Lemma lemma-diff-f proof with the block J: Q x^t - b + S (x^t - y^t) = 0, S = J - Q
    Q, A, xs, b = case()
    Jb = oracle.j_blkdiag(Q, bs)
    J = _block_dense(Jb, Q["n"])
    T = 60
    r = oracle.solve(Q, b, Jblk=Jb, restart=False, maxit=T, stop=oracle.STOP_NONE, trace_iterates=True)
    X, Y = r["trace"]["x"], r["trace"]["y"]
    for t in range(1, T + 1):
        res = A @ X[t] - b + (J - A) @ (X[t] - Y[t])
        assert np.abs(res).max() <= 1e-12 * (1 + np.abs(b).max())


def test_block_j_solves_and_singular_blocks_take_j_diag():
    # a component {0, 1} wholly inside block 0 makes Q^{00} singular with no coupling:
    # that block takes eq. J-diag's diagonal (here diag(2, 2))
    u = [0, 2, 3, 4, 5, 2]
    v = [1, 3, 4, 5, 6, 6]
    Q = synth.from_edges(7, u, v, [1.0] * 6)
    Jb = oracle.j_blkdiag(Q, 2)
    np.testing.assert_array_equal(Jb[0], np.diag(oracle.j_absrowsum(Q)[:2]))
    assert np.linalg.eigvalsh(_block_dense(Jb, 7) - dense.to_dense(Q))[0] >= -1e-12
    b = synth.rhs(Q, synth.uniform(7, 3))
    r = oracle.solve(Q, b, Jblk=Jb, maxit=5000, tol=1e-10)
    assert r["converged"] and r["relres"] <= 1e-10


def test_block_j_converges_on_poisson_like_diagonal_j():
    # Section 4 notes that eq. J-blkdiag performs about as well as eq. J-diag
    Q = synth.poisson2d(16)
    b = synth.rhs(Q, synth.uniform(Q["n"], 5))
    it_d = oracle.solve(Q, b, oracle.j_absrowsum(Q), maxit=5000, tol=1e-10)["iters"]
    for bs in (2, 4, 16):
        r = oracle.solve(Q, b, Jblk=oracle.j_blkdiag(Q, bs), maxit=5000, tol=1e-10)
        assert r["converged"] and 0.5 * it_d <= r["iters"] <= 1.5 * it_d


# --------------------------------------------------------------------------- PCG comparator (Section 4.2)
def test_pcg_matches_scipy_cg_with_jacobi_preconditioner():
    # an independent implementation of the same recurrence: scipy's cg with M^{-1} = diag(Q)^{-1}
    sla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    Q, A = _random_csr(40, 0.2, 12, symmetric=True, spd_shift=0.3)
    b = np.random.default_rng(1).standard_normal(40)
    S = sp.csr_matrix((Q["val"], Q["col"], Q["row_ptr"]), shape=(40, 40))
    Minv = sla.LinearOperator((40, 40), matvec=lambda v: v / np.diag(A))
    xs = []
    sla.cg(S, b, x0=np.zeros(40), rtol=1e-300, atol=0.0, maxiter=8, M=Minv, callback=lambda xk: xs.append(xk.copy()))
    for t in range(1, 9):
        r = oracle.pcg(Q, b, maxit=t, tol=0.0)
        np.testing.assert_allclose(r["x"], xs[t - 1], rtol=1e-11, atol=1e-12)


def test_pcg_finite_termination_with_two_preconditioned_eigenvalues():
    # Q = D^1/2 B D^1/2 with B = (1 - c) I + c 1 1^T (unit diagonal): diag(Q) = D and
    # M^{-1} Q is similar to B, which has two distinct eigenvalues, so PCG terminates
    # after 2 iterations (a dropped beta, sign or preconditioner step would not)
    n, c = 30, 0.3
    d = np.random.default_rng(2).uniform(0.5, 4.0, n)
    B = (1 - c) * np.eye(n) + c * np.ones((n, n))
    A = np.sqrt(d)[:, None] * B * np.sqrt(d)[None, :]
    Q = _dense_to_csr(A)
    b = np.random.default_rng(3).standard_normal(n)
    r = oracle.pcg(Q, b, maxit=50, tol=1e-12)
    assert r["iters"] == 2
    np.testing.assert_allclose(r["x"], np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("case", [_tiny_spd, _tiny_laplacian])
def test_pcg_recursive_residual_tracks_true_residual(case):
    Q, A, xs, b = case()
    for t in (5, 15, 25):
        r = oracle.pcg(Q, b, maxit=t, tol=0.0)
        true = np.linalg.norm(b - A @ r["x"])
        assert abs(r["rr"][-1] - true) <= 1e-10 * np.linalg.norm(b)
    r = oracle.pcg(Q, b, maxit=500, tol=1e-12)
    assert np.linalg.norm(A @ r["x"] - b) <= 1e-11 * np.linalg.norm(b)


def test_openmp_timing_build_computes_the_same_bits():
    # the CPU baseline times the -O3 -fopenmp build of the same source: it
    # spreads independent rows over threads and keeps every sum in one thread
    Q, b, _ = synth.workload("poisson3d_20")
    J = oracle.j_absrowsum(Q)
    a = oracle.solve(Q, b, J, maxit=150, stop=oracle.STOP_NONE, trace=True)
    c = oracle.solve(Q, b, J, maxit=150, stop=oracle.STOP_NONE, trace=True, omp=True)
    np.testing.assert_array_equal(a["x"], c["x"])
    np.testing.assert_array_equal(a["trace"]["d"], c["trace"]["d"])
    assert a["restarts"] == c["restarts"] and oracle.host_cores() >= 1
