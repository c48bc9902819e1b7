"""Compile the FP64 C oracle into a shared object (test infrastructure only).

The oracle is plain C99 with optional OpenMP.  It is compiled without FMA
contraction (-ffp-contract=off) so that its results are the same on x86-64 and
AArch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbem_oracle.c")
LIB = os.path.join(HERE, "liblbem_oracle.so")


def build(force: bool = False) -> str:
    """Build liblbem_oracle.so next to its source if it is missing or stale."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
