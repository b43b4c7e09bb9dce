"""Compile the C oracle into oracle/_build/liboracle.so (test infrastructure).

Plain gcc, -O2, no fast-math and no FMA contraction, so the oracle's rounding
is the plain IEEE double evaluation of the code as written.  A second build,
liboracle_omp.so, adds -fopenmp (independent nodes in parallel, the same
per-node arithmetic) for the CPU-baseline timing on all host cores.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = os.path.join(HERE, "lbm_oracle.c")


LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def _build_one(lib, extra, force):
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(SRC[:-1] + "h"))):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas"] + extra + ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


def build(force=False):
    return _build_one(LIB, [], force)


def build_omp(force=False):
    """The OpenMP build, or None where the compiler has no OpenMP."""
    try:
        return _build_one(LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        return None


if __name__ == "__main__":
    print(build(force=True), build_omp(force=True))
