"""Compile the CPU oracle (test infrastructure; see ccg_oracle.cpp).

Plain g++, serial code, IEEE semantics (no fast-math).  -fcx-fortran-rules
gives complex multiplication the Fortran definition (no C99 Annex G NaN
recovery), which is the arithmetic of the FORTRAN90 library the oracle
stands in for.

Two builds of the same source: liboracle.so (serial; the tests' oracle) and
liboracle_omp.so (-fopenmp: the dense operator's independent output
elements on all allowed host cores, bit-identical results; the all-core CPU
baseline of the benchmark).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ccg_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def _compile(out, extra, force):
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fcx-fortran-rules"] + extra + ["-shared", "-fPIC", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force=False):
    """Build oracle/_build/liboracle.so if it is missing or older than its source."""
    return _compile(LIB, [], force)


def build_omp(force=False):
    """Build oracle/_build/liboracle_omp.so (OpenMP); raises if the compiler
    has no OpenMP support."""
    return _compile(LIB_OMP, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_omp(force=True))
