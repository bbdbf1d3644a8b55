"""Compile the C oracle into oracle/_build/liboracle.so with gcc.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline leg load the result. -ffp-contract=off keeps gcc from fusing a
multiply into an add (aarch64 gcc does so by default in GNU C mode), so every
rounding is the one written in oracle.c.
"""

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
HDR = os.path.join(HERE, "oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", "-Wall", "-Wextra", "-Wno-unused-parameter"]


def build(force=False):
    """The loops over particles run on OpenMP threads when gcc supports it
    (or_set_threads; one thread unless raised); without it the same source
    builds single-threaded."""
    os.makedirs(OUT_DIR, exist_ok=True)
    fresh = os.path.exists(LIB) and all(
        os.path.getmtime(LIB) >= os.path.getmtime(p) for p in (SRC, HDR, __file__))
    if fresh and not force:
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    try:
        subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, SRC, "-lm"],
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
