"""Compile the plain C oracle into ``oracle/liboracle.so`` with gcc.

Test infrastructure: the oracle is a checker, never part of the product path.
``-frounding-math`` keeps the directed-rounding interval walk honest and
``-ffp-contract=off`` forbids fused multiply-adds (aarch64 gcc fuses by
default), so the FP64 and interval sequences are the ones the source spells.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

FLAGS = ["-O1", "-std=c11", "-fPIC", "-shared", "-frounding-math", "-ffp-contract=off",
         "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", *FLAGS, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
