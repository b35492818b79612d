"""Compile the CPU oracle (test infrastructure; see ccg_oracle.cpp).

Plain g++, serial code, IEEE semantics (no fast-math).  -fcx-fortran-rules
gives complex multiplication the Fortran definition (no C99 Annex G NaN
recovery), which is the arithmetic of the FORTRAN90 library the oracle
stands in for.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ccg_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force=False):
    """Build oracle/_build/liboracle.so if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fcx-fortran-rules", "-shared", "-fPIC", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
