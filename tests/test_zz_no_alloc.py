"""GPU check of aj_solve_noalloc, the allocation-free solve.

Some callers cannot allocate device memory: a service whose other streams
must not stall on the device synchronisation of cudaMalloc / cudaFree, or a
process whose device memory a framework's caching allocator has reserved up
front.  aj_solve_noalloc takes its scratch from one fixed device array inside
libaj instead.  These tests call it through the C ABI and compare its output
with the ordinary entry point (aj_create + aj_set + aj_solve) on the same
system: twice in a row, because every call reuses the same array and must
start clean.  The tolerance is the FP64 iterate-parity bound used by the other
GPU tests.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2407_03272_gb300 import aj  # noqa: E402

REL = 1e-10
GRID = 16  # the 64 x 64 system has 16 tiles of 256 rows


def _device_system(name):
    Q, b, _ = synth.workload(name)
    dev = torch.device("cuda", 0)
    t = [torch.from_numpy(np.ascontiguousarray(a)).to(dev)
         for a in (Q["row_ptr"], Q["col"], Q["val"], b)]
    return Q, b, t


def _reference(Q, b, **kw):
    # the ordinary entry point in the configuration the allocation-free one
    # runs: CSR rows, the stored sweep form, the same grid (so the FP64
    # reductions are summed in the same order)
    ctx = aj.from_csr(Q, b, device="cuda:0")
    ctx.set(format=aj.AJ_FMT_CSR, sweep_form=aj.AJ_SWEEP_STORED, grid_ctas=GRID, **kw)
    x, info = ctx.solve()
    ctx.close()
    return x, info


def _noalloc(t, n, **kw):
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda:0")
    st, info = aj.solve_noalloc(*t, out, stream=torch.cuda.current_stream(), grid_ctas=GRID, **kw)
    torch.cuda.synchronize()
    return st, out.cpu().numpy(), info


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_matches_solve_fixed_iterations_twice():
    torch.cuda.set_device(0)
    Q, b, t = _device_system("poisson2d_64")
    T = 200
    ref, rinfo = _reference(Q, b, stop=aj.AJ_STOP_NONE, maxit=T)
    for _ in range(2):
        st, x, info = _noalloc(t, Q["n"], stop=aj.AJ_STOP_NONE, maxit=T)
        assert st == aj.AJ_EMAXIT and info["iters"] == T
        assert info["restarts"] == rinfo["restarts"]
        assert _rel(x, ref) <= REL


def test_noalloc_matches_solve_to_tolerance_twice():
    torch.cuda.set_device(0)
    Q, b, t = _device_system("poisson2d_64")
    ref, rinfo = _reference(Q, b, tol=1e-8, maxit=20000)
    assert rinfo["status"] == aj.AJ_OK
    for _ in range(2):
        st, x, info = _noalloc(t, Q["n"], tol=1e-8, maxit=20000)
        assert st == aj.AJ_OK and info["status"] == aj.AJ_OK
        assert info["iters"] == rinfo["iters"]
        assert info["relres"] <= 1e-8
        assert info["relres"] == rinfo["relres"] or abs(info["relres"] - rinfo["relres"]) <= 1e-3 * rinfo["relres"]
        assert _rel(x, ref) <= REL


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    torch.cuda.set_device(0)
    n = aj.AJ_NOALLOC_MAX_N + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda:0")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    v = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    b = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    st, _ = aj.solve_noalloc(rp, ci, v, b, out)
    assert st == aj.AJ_ENOMEM
