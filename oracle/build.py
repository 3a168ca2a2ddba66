"""Build the FP64 CPU oracle library (test infrastructure only).

Compiles ``colatus_oracle.c`` into ``libcolatus_oracle.so`` next to this file
with plain IEEE double arithmetic (no fast-math, no FMA contraction) and
OpenMP over independent target rows.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "colatus_oracle.c")
LIB = os.path.join(HERE, "libcolatus_oracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
