"""Build step of the oracle's C core (plain C, FP64, OpenMP).

TEST INFRASTRUCTURE ONLY: the library built here is loaded by the tests, the
smoke check and the benchmark's CPU-baseline leg, never by the product path.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "lattice_oracle.c")
LIB = os.path.join(BUILD, "liboracle.so")


def build(force=False):
    """Compile lattice_oracle.c into _build/liboracle.so (no -ffast-math, so
    the FP64 arithmetic is plain IEEE)."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
