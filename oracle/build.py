"""Compiles the FP64 CPU oracle (fmm_oracle.c) into oracle/_fmm_oracle.so.

Test infrastructure: the library is loaded only by the tests, the smoke check
and the CPU-baseline leg of the benchmark.  Built with -ffp-contract=off so
that the canonical single-precision coordinate map is evaluated with one
rounding per operation on every host (aarch64 gcc contracts a*b+c by default).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fmm_oracle.c")
LIB = os.path.join(HERE, "_fmm_oracle.so")


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
