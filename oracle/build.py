"""Compile the plain-C oracle into oracle/_build/liboracle.so (gcc, no CUDA).

Flags follow the paper-silent rounding reading: no floating-point contraction, IEEE
sqrt and division (-O2 -ffp-contract=off, no -ffast-math).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force=False):
    """Build liboracle.so if it is missing or older than its source; return its path.
    OpenMP (the all-core timing of the CPU baseline) is used when the compiler has it;
    otherwise the library is built without it and runs one thread."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(__file__))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC",
            "-shared", "-o", tmp, SRC, "-lm"]
    if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
