"""Compile the C part of the oracle (the direct sum) into oracle/_direct.so.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain gcc, -O2, IEEE
arithmetic (no -ffast-math), OpenMP for the row loop.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "direct.c")
LIB = os.path.join(HERE, "_direct.so")


def build_oracle(force=False):
    """Build oracle/_direct.so if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB
