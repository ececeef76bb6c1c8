"""Build the CPU oracle shared libraries (test infrastructure only).

Compiles ``dgsem_oracle.cpp`` with g++ (OpenMP, no FMA contraction so that
the arithmetic order is the one written in the source) twice:
``oracle/_build/libdgsem_oracle.so`` with double arithmetic (the FP64
oracle) and ``libdgsem_oracle_ext.so`` with long double (extended
precision: 64-bit significand on x86-64, 113-bit on aarch64), the parity
reference whose own rounding error is far below the FP64 tolerance.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dgsem_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdgsem_oracle.so")
LIB_EXT = os.path.join(OUT_DIR, "libdgsem_oracle_ext.so")


def _compile(out, defines, force):
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off",
           "-fPIC", "-shared"] + defines + [SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False, extended: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if extended:
        return _compile(LIB_EXT, ["-DORA_REAL=long double"], force)
    return _compile(LIB, [], force)


def build_all(force: bool = False):
    return build(force), build(force, extended=True)


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv))
