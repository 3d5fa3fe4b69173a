"""GPU checks of the continuous-batching server (aj_server_*).

* Alone equals in the mix: every request solved by the server, while other
  requests of other sizes share the GPU, queue for memory and arrive during
  its run, returns exactly what aj_solve returns for the same system alone
  with the same gang size (grid_ctas) -- bitwise, in FP64 and in the FP32
  refinement mode.
* The server keeps its admitted device memory within the budget, holds
  several requests at once, and rejects a request larger than the budget.
* Without a fixed gang size every result still meets its FP64 tolerance.
"""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402


def _mix(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        kind = k % 3
        if kind == 0:
            Q = synth.poisson2d(int(rng.integers(6, 64)))
        elif kind == 1:
            Q = synth.rgg_knn_laplacian(int(rng.integers(300, 3000)), seed=300 + k)
        else:
            Q = synth.chung_lu_laplacian(int(rng.integers(500, 4000)), seed=400 + k, mean_degree=6.0)
        nrhs = int(rng.integers(1, 4))
        B = np.stack([synth.rhs(Q, synth.uniform(Q["n"], 2000 * k + r)) for r in range(nrhs)], axis=1)
        out.append((Q, B))
    return out


def _cm(B):
    return np.ascontiguousarray(B.T).reshape(-1)


def _solo(Q, B, **kw):
    ctx = aj.from_csr(Q, _cm(B), nrhs=B.shape[1])
    ctx.set(**kw)
    x, info = ctx.solve()
    ctx.close()
    return x, info


@pytest.mark.parametrize("precision", ["fp64", "fp32_ir"])
def test_alone_equals_in_the_mix(precision):
    torch.cuda.set_device(0)
    mix = _mix(21, seed=7)
    kw = dict(precision=precision, tol=1e-9, maxit=40000)
    gangs = [1 + (k % 3) for k in range(len(mix))]
    # a budget that admits a few requests at a time, so that later ones queue
    sizes = [(Q["n"], int(Q["row_ptr"][-1])) for Q, _ in mix]
    budget = int(6 * max(n * 8 * 30 + z * 20 for n, z in sizes)) + (8 << 20)
    srv = aj.Server(budget, max_slots=6)
    tickets = []
    half = len(mix) // 2
    for k in range(half):
        Q, B = mix[k]
        tickets.append(srv.submit_csr(Q, _cm(B), nrhs=B.shape[1], grid_ctas=gangs[k], **kw))
    time.sleep(0.05)  # the rest arrives while the first half is on the GPU
    for k in range(half, len(mix)):
        Q, B = mix[k]
        tickets.append(srv.submit_csr(Q, _cm(B), nrhs=B.shape[1], grid_ctas=gangs[k], **kw))
    results = [srv.result(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(mix)
    assert stats["peak_active"] >= 2
    assert stats["peak_bytes"] <= budget
    for (Q, B), g, (st, x, info) in zip(mix, gangs, results):
        assert st == aj.AJ_OK, info
        xs, sinf = _solo(Q, B, grid_ctas=g, **kw)
        assert info["iters"] == sinf["iters"]
        np.testing.assert_array_equal(x, xs)


def test_server_default_gangs_meet_tolerance_and_existing_contexts():
    torch.cuda.set_device(0)
    mix = _mix(12, seed=8)
    srv = aj.Server(8 << 30, max_slots=64)
    tickets = []
    ctxs = []
    for k, (Q, B) in enumerate(mix):
        if k % 2:
            tickets.append(srv.submit_csr(Q, _cm(B), nrhs=B.shape[1], tol=1e-8, maxit=40000))
        else:
            c = aj.from_csr(Q, _cm(B), nrhs=B.shape[1])
            c.set(tol=1e-8, maxit=40000)
            ctxs.append(c)
            tickets.append(srv.submit(c))
    for (Q, B), t in zip(mix, tickets):
        st, x, info = srv.result(t)
        assert st == aj.AJ_OK
        X = x.reshape(B.shape[1], Q["n"]).T
        for r in range(B.shape[1]):
            rel = np.linalg.norm(B[:, r] - oracle.spmv(Q, X[:, r])) / np.linalg.norm(B[:, r])
            assert rel <= 1e-8
    srv.close()


def test_server_rejects_request_larger_than_budget():
    torch.cuda.set_device(0)
    Q = synth.poisson2d(64)
    b = synth.rhs(Q, synth.uniform(Q["n"], 1))
    srv = aj.Server(1 << 16, max_slots=4)
    with pytest.raises(aj.AJError) as e:
        srv.submit_csr(Q, b)
    assert e.value.status == aj.AJ_EBUSY
    srv.close()
