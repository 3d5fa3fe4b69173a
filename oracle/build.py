"""Compile the plain-C FP64 oracle into oracle/_build/liboracle.so, and the
same source with OpenMP into oracle/_build/liboracle_omp.so.

Test infrastructure: building the oracle is not running it.  -ffp-contract=off
keeps a*b+c as two roundings on every host (aarch64 gcc would otherwise fuse
it), so the oracle gives the same bits on x86-64 and arm64.  The OpenMP build
(-O3 -fopenmp) serves only the CPU baseline timings: it spreads the rows of a
product and the element-wise updates over the host's cores and keeps every
sum in one thread in index order, so it computes the same bits.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aj_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def _compile(lib, flags, force):
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + flags + ["-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                             "-std=c11", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """The correctness oracle: one thread, -O2."""
    return _compile(LIB, ["-O2", "-Wno-unknown-pragmas"], force)


def build_omp(force: bool = False) -> str:
    """The baseline timing build: -O3 -fopenmp, the same bits."""
    return _compile(LIB_OMP, ["-O3", "-fopenmp"], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
