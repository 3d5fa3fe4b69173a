"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point that include/aj.h declares.  No GPU work is issued."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2407_03272_gb300 import aj

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "aj.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(aj_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("aj_create", "aj_set", "aj_set_stream", "aj_solve", "aj_solve_batch",
                 "aj_server_create", "aj_submit", "aj_poll", "aj_get_state", "aj_set_state",
                 "aj_destroy", "aj_server_destroy", "aj_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = aj.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert {s[0] for s in aj.SIGNATURES} == set(declared_functions())


def test_defaults_and_strings():
    p = aj.params()
    assert p.j_policy == aj.AJ_J_ABSROWSUM and p.restart == aj.AJ_RESTART_ADAPTIVE
    assert p.K0 == 2 and p.tol == 1e-8 and p.momentum == 1 and p.precision == aj.AJ_FP64
    L = aj.lib()
    for st in (0, -1, -2, -3, -4, -5, -6, -7, -8, 1):
        assert L.aj_strerror(st)
    assert L.aj_strerror(12345) == b"unknown status"


def test_null_arguments_rejected_without_gpu_work():
    L = aj.lib()
    out = ctypes.c_void_p()
    assert L.aj_create(None, None, 1, ctypes.byref(out)) == aj.AJ_EINVAL
    csr = aj.aj_csr(4, 0, None, None, None, 0)
    assert L.aj_create(ctypes.byref(csr), None, 1, ctypes.byref(out)) == aj.AJ_EINVAL
    csr = aj.aj_csr(0, 0, None, None, None, 0)
    assert L.aj_create(ctypes.byref(csr), None, 5, ctypes.byref(out)) == aj.AJ_EINVAL
    assert L.aj_set(None, None) == aj.AJ_EINVAL
    assert L.aj_solve(None, None, 0, None) == aj.AJ_EINVAL
    cnt = ctypes.c_int64()
    assert L.aj_restart_log(None, 0, None, 0, ctypes.byref(cnt)) == aj.AJ_EINVAL
    s = ctypes.c_void_p()
    assert L.aj_server_create(0, 1, ctypes.byref(s)) == aj.AJ_EINVAL


def test_struct_layouts_match_header():
    # sizes a C compiler gives the three public structs on LP64
    assert ctypes.sizeof(aj.aj_csr) == 48
    assert ctypes.sizeof(aj.aj_info) == 88
    assert ctypes.sizeof(aj.aj_params) == 144
    assert ctypes.sizeof(aj.aj_tuning) == 56


def test_failure_hooks_validate_their_arguments_without_gpu_work():
    L = aj.lib()
    assert L.aj_test_barrier_stall(-2, 1.0) == aj.AJ_EINVAL
    assert L.aj_test_barrier_stall(0, 0.0) == aj.AJ_EINVAL
    assert L.aj_test_barrier_stall(0, 5000.0) == aj.AJ_EINVAL
    assert L.aj_test_barrier_stall(-1, 1.0) == aj.AJ_OK   # disarm
    assert L.aj_test_alloc_fail(-2) == aj.AJ_EINVAL
    assert L.aj_test_alloc_fail(-1) == aj.AJ_OK          # disarm


def test_noalloc_binding_refuses_bad_arrays_before_the_call():
    torch = pytest.importorskip("torch")
    n = 5
    rp = torch.arange(n + 1, dtype=torch.int32)
    ci = torch.arange(n, dtype=torch.int32)
    v = torch.ones(n, dtype=torch.float64)
    b = torch.ones(n, dtype=torch.float64)
    out = torch.zeros(n, dtype=torch.float64)
    bad = [
        dict(row_ptr=rp.to(torch.int64)),                 # int64 row pointers
        dict(col=ci.to(torch.int64)),
        dict(val=v.to(torch.float32)),
        dict(b=b.to(torch.float32)),                      # float32 right-hand side
        dict(x_out=torch.zeros(n - 1, dtype=torch.float64)),  # short output
        dict(b=torch.ones(n - 2, dtype=torch.float64)),
        dict(val=torch.ones(n + 1, dtype=torch.float64)),  # val and col differ
        dict(x_out=np.zeros(n)),                           # not a tensor
    ]
    base = dict(row_ptr=rp, col=ci, val=v, b=b, x_out=out)
    for case in bad:
        args = dict(base, **case)
        with pytest.raises(ValueError):
            aj.solve_noalloc(args["row_ptr"], args["col"], args["val"], args["b"], args["x_out"])
    with pytest.raises(ValueError):
        aj.solve_noalloc(rp, ci, v, b, out, x0=torch.zeros(n, dtype=torch.float32))
    # well-formed host tensors are refused too: the entry point takes device arrays
    with pytest.raises(ValueError, match="device"):
        aj.solve_noalloc(rp, ci, v, b, out)


def test_cache_stats_without_gpu_work():
    s = aj.cache_stats()
    assert set(s) == {"order_hits", "order_misses", "tune_hits", "tune_misses"}
    assert all(v >= 0 for v in s.values())
