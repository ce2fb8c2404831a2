"""Compile the CPU oracle (plain C, double precision) into oracle/_build/liboracle.so.

The oracle is test infrastructure: it is built here so that the test-suite,
the smoke check and the benchmark's CPU baseline can load it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC_OMP = os.path.join(HERE, "oracle_omp.c")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")
# -ffp-contract=off: no fused multiply-add, so the oracle rounds the same
# way on every host architecture.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def _stale(lib, *srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(LIB, SRC):
        subprocess.check_call(["gcc", *CFLAGS, "-o", LIB + ".tmp", SRC, "-lm"])
        os.replace(LIB + ".tmp", LIB)
    return LIB


def build_omp(force: bool = False) -> str:
    """The multi-core CPU baseline (oracle_omp.c, the oracle's element
    arithmetic with its loops split over OpenMP threads)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(LIB_OMP, SRC, SRC_OMP):
        subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", LIB_OMP + ".tmp", SRC_OMP, "-lm"])
        os.replace(LIB_OMP + ".tmp", LIB_OMP)
    return LIB_OMP


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
