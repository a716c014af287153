"""Build the CPU oracle shared library (test infrastructure only).

gcc, C11, no FMA contraction (the oracle's fused multiply-adds are the explicit
fma()/fmaf() calls of its decision arithmetic), OpenMP over particles in the
partner search (the paper's own shared-memory scheme parallelises that loop).
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kmc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def _x86_fma_flags():
    """On x86-64 CPUs with FMA, let gcc inline the oracle's explicit fma()
    calls (same IEEE result as the libm call, much faster).  aarch64 has them
    natively."""
    if platform.machine() not in ("x86_64", "AMD64"):
        return []
    try:
        flags = open("/proc/cpuinfo").read()
    except OSError:
        return []
    return ["-mfma"] if " fma" in flags else []


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "kmc_oracle.h"))
    ):
        return LIB
    cmd = [
        "gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
        "-ffp-contract=off", "-fno-fast-math", *_x86_fma_flags(), "-o", LIB, SRC, "-lm",
    ]
    subprocess.check_call(cmd, cwd=HERE)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
