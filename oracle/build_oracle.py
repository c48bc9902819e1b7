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
LIB32 = os.path.join(HERE, "liblbem_oracle_f32.so")


def build(force: bool = False, fp32: bool = False) -> str:
    """Build liblbem_oracle.so (FP64, the oracle) next to its source if it is missing or stale.  fp32=True builds
    liblbem_oracle_f32.so instead: the same source with every quantity in float (and single-precision constants),
    used only to time a like-for-like CPU figure."""
    lib = LIB32 if fp32 else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    extra = ["-DOR_REAL=float", "-fsingle-precision-constant"] if fp32 else []
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp"] + extra + [SRC, "-o", tmp,
                                                                                                   "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, fp32=True))
