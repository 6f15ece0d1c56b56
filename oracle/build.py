"""Compiles the FP64 oracle (plain C) into oracle/libgencd_oracle.so with gcc.

Test infrastructure: the library is loaded only by the tests, the smoke check
and the benchmark's CPU-baseline leg.  No FMA contraction, no fast-math, so that
results are identical on x86-64 and aarch64 hosts.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gencd_oracle.c")
LIB = os.path.join(HERE, "libgencd_oracle.so")


OMP_SRC = os.path.join(HERE, "gencd_omp.c")
OMP_LIB = os.path.join(HERE, "libgencd_omp.so")


def build_omp(force: bool = False) -> str:
    """The OpenMP baseline of Section 4.2 (gencd_omp.c linked with the
    oracle), compiled with -fopenmp into oracle/libgencd_omp.so."""
    deps = [OMP_SRC, SRC, os.path.join(HERE, "gencd_omp.h"), os.path.join(HERE, "gencd_oracle.h")]
    if not force and os.path.exists(OMP_LIB) and os.path.getmtime(OMP_LIB) >= max(os.path.getmtime(d) for d in deps):
        return OMP_LIB
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wextra", "-o", OMP_LIB + ".tmp", OMP_SRC, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(OMP_LIB + ".tmp", OMP_LIB)
    return OMP_LIB


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gencd_oracle.h"))):
        return LIB
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wextra", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
