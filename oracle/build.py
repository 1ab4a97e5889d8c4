"""Compile the C half of the oracle into oracle/libftlm_oracle.so.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain gcc, no -march flags,
so the same source builds on x86-64 and on Arm hosts; -ffp-contract=off keeps the
arithmetic exactly as written (no fused multiply-adds on hosts that contract by
default).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ftlm_oracle.c")
LIB = os.path.join(HERE, "libftlm_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
