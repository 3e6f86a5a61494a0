"""Build the CPU oracle (plain C, FP64) into oracle/_build/liboracle.so.

Test infrastructure only: the oracle checks the CUDA library and is never part of
its compute path.  Compiled with IEEE semantics (no fast-math, no FMA
contraction) so that x86-64 and aarch64 builds compute the same way.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = os.path.join(HERE, "gp_oracle.c")


def build(force: bool = False) -> str:
    """Compile the oracle if needed; return the path of the shared library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gp_oracle.h"))
    ):
        return LIB
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm"]
    try:  # OpenMP only parallelises independent line solves; results do not change
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
