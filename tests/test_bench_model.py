"""CPU checks of the benchmark's byte and instruction model: the per-sweep
figures that every reported GB/s and roofline fraction divides by."""
import importlib.util
import os

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_poisson_sizes_and_headline_bytes():
    b = _bench()
    # 7-point Dirichlet Poisson on N^3: nnz = 7 n - 6 N^2
    for N in (3, 4, 9):
        Q = synth.poisson3d(N)
        assert Q["n"] == N ** 3 and int(Q["row_ptr"][-1]) == 7 * N ** 3 - 6 * N ** 2
    n, nnz = 256 ** 3, 7 * 256 ** 3 - 6 * 256 ** 2
    assert nnz == 117047296
    # the method's minimum: values + int32 columns, the row pointers, 5 n-vectors
    assert b.algorithmic_bytes(n, nnz, "fp64") == nnz * 12 + 4 * (n + 1) + 5 * 8 * n == 2142765060
    assert b.algorithmic_bytes(n, nnz, "fp32_ir") == nnz * 8 + 4 * (n + 1) + 5 * 4 * n
    assert b.algorithmic_bytes(n, nnz, "bf16_ir") == nnz * 6 + 4 * (n + 1) + 5 * 4 * n
    # the sweep forms' own traffic: stored keeps Q x (two more vectors), the
    # difference form one more again
    assert b.algorithmic_bytes(n, nnz, "fp64", "stored") - b.algorithmic_bytes(n, nnz, "fp64") == 2 * 8 * n
    assert b.algorithmic_bytes(n, nnz, "fp64", "delta") - b.algorithmic_bytes(n, nnz, "fp64") == 3 * 8 * n


def test_stencil_and_several_rhs_bytes():
    b = _bench()
    n, nnz = 1000, 4960
    # the stencil format reads no matrix: the vectors alone
    assert b.algorithmic_bytes(n, nnz, "fp32_ir", stencil=True) == 5 * 4 * n
    # right-hand sides share one pass over the matrix
    one = b.algorithmic_bytes(n, nnz, "fp64")
    four = b.algorithmic_bytes(n, nnz, "fp64", nrhs=4)
    assert four - one == 3 * 5 * 8 * n


def test_fp64_instruction_model():
    b = _bench()
    n, nnz = 10, 64
    # one FMA per stored entry plus the per-row update and reductions
    assert b.fp64_ops(n, nnz, "delta") == nnz + 8 * n
    assert b.fp64_ops(n, nnz, "stored") == nnz + 9 * n
    assert b.fp64_ops(n, nnz, "lazy") == 2 * nnz + 11 * n
    assert b.fp64_ops(n, nnz, "y") == nnz + 4.25 * n
    # the measured FP64 issue peak: 2 instructions per clock on 152 SMs at 2.06 GHz
    assert abs(b.FP64_PEAK_TOPS - 152 * 2 * 2.06e9 / 1e12) < 1e-3
