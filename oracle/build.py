"""Compile the plain-C oracle (``oracle.c``) into ``_build/liboracle.so``.

Test infrastructure: the GPU library never builds, links or loads this.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.c")
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(src)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src]
    # OpenMP for the loops over independent columns (same arithmetic per
    # column); without a usable OpenMP runtime the oracle builds serial
    r = subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + ["-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
