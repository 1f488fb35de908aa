"""Compile the C oracle into oracle/liboracle.so (test infrastructure only).

gcc, -O2, single translation unit, -ffp-contract=off so that the double
arithmetic of the SIR threshold tables is exactly the sequence of IEEE
operations written in the source (no fused multiply-adds).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "amb_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False):
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-Wall", "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
