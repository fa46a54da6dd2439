"""Compile the plain-C oracle into ``oracle/liblsq_oracle.so``.

Test infrastructure only: the oracle is built (never used) by the package
build step so that the tests and the benchmark's CPU-baseline leg find it.
``-ffp-contract=off`` keeps every product and sum separately rounded on both
x86-64 and AArch64, so the oracle gives identical bits on x86 and Arm.
``-fopenmp`` spreads loops with independent iterations over the host cores;
every sum keeps its order, so the bits do not depend on the thread count.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lsq_oracle.c")
LIB = os.path.join(HERE, "liblsq_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-frounding-math", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
