"""Compiles the CPU oracle (oracle.c) into liboracle.so next to this file.

Flags: -O2 -ffp-contract=off (no FMA contraction, no fast-math) so every
floating-point operation in oracle.c is one IEEE FP64 operation, in the order
written.  -fopenmp: the loops over cells and elements can be shared among
threads (oracle.set_threads; one thread unless set), without changing any
element's operations or their order.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-fopenmp", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
