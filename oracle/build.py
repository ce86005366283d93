"""Compile the CPU oracle (phs_oracle.c) into oracle/liboracle.so with gcc.

TEST INFRASTRUCTURE: the oracle is only loaded by the tests, the smoke check and
the benchmark's CPU-baseline leg.  -ffp-contract=off keeps every squared
distance as dx*dx + dy*dy with two roundings, the arithmetic the bit-exact
neighbour comparisons assume.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "phs_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
