"""Compile the oracle's C loops into oracle/_lib/liboracle.so with gcc.

Building the checker is part of `__graft_entry__.build()`; building is not using it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_lib", "liboracle.so")
SRC = os.path.join(HERE, "smg_oracle.c")


def build(force=False):
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    # -O2 without -ffast-math: IEEE semantics, evaluation order as written.
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


OMP_LIB = os.path.join(HERE, "_lib", "liboracle_omp.so")
OMP_SRC = os.path.join(HERE, "smg_omp.c")


def build_omp(force=False):
    """The multicolour OpenMP loops (all-cores CPU baseline), same flags plus -fopenmp."""
    os.makedirs(os.path.dirname(OMP_LIB), exist_ok=True)
    if not force and os.path.exists(OMP_LIB) and os.path.getmtime(OMP_LIB) >= os.path.getmtime(OMP_SRC):
        return OMP_LIB
    tmp = OMP_LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           OMP_SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OMP_LIB)
    return OMP_LIB


if __name__ == "__main__":
    print(build(force=True))
    print(build_omp(force=True))
