"""GPU checks of the PCG comparator (aj_pcg_solve): conjugate gradients with
M = diag(Q), Sec. 4.2's main competitor, against the oracle's PCG (Saad's
Alg. 9.1 in plain C)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402


def _run(Q, b, **kw):
    c = aj.from_csr(Q, b)
    c.set(**kw)
    return c, c.pcg_solve()


@pytest.mark.parametrize("case", ["poisson2d_64", "poisson3d_17", "graph", "sdd"])
def test_pcg_iterates_match_oracle(case):
    if case == "graph":
        Q = synth.chung_lu_laplacian(6000, seed=11, mean_degree=8.0)  # hubs: warp-per-row sums
    elif case == "sdd":
        Q = synth.sdd(700)
    elif case == "poisson3d_17":
        Q = synth.poisson3d(17)
    else:
        Q, _, _ = synth.workload(case)
    b = synth.rhs(Q, synth.uniform(Q["n"], 9))
    # on the SDD matrix M^{-1} Q has two distinct eigenvalues: CG is exact after
    # two iterations and a third divides 0 by 0 (in the oracle too)
    for T in ((1, 2) if case == "sdd" else (1, 7, 40)):
        _, (x, info) = _run(Q, b, tol=0.0, maxit=T)
        ref = oracle.pcg(Q, b, maxit=T, tol=0.0)
        assert info["iters"] == ref["iters"] == T
        assert np.linalg.norm(x - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("case", ["poisson3d_24", "graph"])
def test_pcg_solves_to_tolerance_like_the_oracle(case):
    if case == "graph":
        Q = synth.rgg_knn_laplacian(20000, seed=3)
    else:
        Q = synth.poisson3d(24)
    b = synth.rhs(Q, synth.uniform(Q["n"], 4))
    _, (x, info) = _run(Q, b, tol=1e-8, maxit=20000)
    ref = oracle.pcg(Q, b, maxit=20000, tol=1e-8)
    assert info["status"] == aj.AJ_OK
    # the recursive residual crosses 1e-8 at the same iteration, give or take one
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert info["relres"] <= 1.01e-8
    assert abs(info["relres"] - np.linalg.norm(b - oracle.spmv(Q, x)) / np.linalg.norm(b)) <= 1e-12


def test_pcg_x0_maxit_and_refusals():
    Q = synth.poisson2d(40)
    b = synth.rhs(Q, synth.uniform(Q["n"], 2))
    x0 = synth.uniform(Q["n"], 3)
    _, (x, info) = _run(Q, b, tol=0.0, maxit=12, x0=x0)
    ref = oracle.pcg(Q, b, maxit=12, tol=0.0, x0=x0)
    assert np.linalg.norm(x - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])
    _, (_, info) = _run(Q, b, tol=1e-14, maxit=3)
    assert info["status"] == aj.AJ_EMAXIT and info["iters"] == 3
    # zero right-hand side: x = 0 at once
    _, (x, info) = _run(Q, np.zeros(Q["n"]), tol=1e-8, maxit=100)
    assert info["iters"] == 0 and not x.any()
    # several right-hand sides are refused
    c = aj.from_csr(Q, np.concatenate([b, b]), nrhs=2)
    c.set()
    with pytest.raises(RuntimeError):
        c.pcg_solve(out=np.empty(2 * Q["n"]))
