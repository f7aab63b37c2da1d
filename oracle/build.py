"""Compile the CPU oracle (``rdo.c``) into ``liboracle.so`` beside it.

Test infrastructure: the oracle is built so that the tests, the smoke check
and the benchmark's CPU-baseline leg can load it; the product library never
links or loads it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rdo.c")
HDR = os.path.join(HERE, "rdo.h")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = [
    "-O2",
    "-std=gnu11",
    "-fPIC",
    "-shared",
    # every float operation rounds exactly where the source says it does
    "-ffp-contract=off",
    "-fno-fast-math",
    "-Wall",
]


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
