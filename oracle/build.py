"""Compile the C oracle (oracle/hgks_ref.c) into oracle/_build/libhgks_ref.so.

Test infrastructure only.  Plain gcc, FP64, no FMA contraction (so x86 and Arm
builds round identically apart from libm), OpenMP over interfaces only.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hgks_ref.c")
HDR = os.path.join(HERE, "hgks_ref.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhgks_ref.so")


def compile_oracle(src, out):
    """Compile one oracle source file into the shared library `out` (the
    header is found beside `src` or in this folder)."""
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-I", HERE, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_oracle(force=False):
    """Build the oracle shared library if missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(LIB) for p in (SRC, HDR))
    if stale:
        compile_oracle(SRC, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
