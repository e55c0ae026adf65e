"""Compile the oracle's C source into a shared library (test infrastructure only).

Built with ``-O2 -ffp-contract=off`` so the compiler fuses no multiply-add:
the oracle's arithmetic is exactly the operations written in ``pf_oracle.c``.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pf_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def build(force=False, openmp=False):
    """Compile ``liboracle.so`` (or, openmp=True, ``liboracle_omp.so``: the
    same source with its RHS loop shared among the host cores, used only for
    the timed all-core CPU baseline) if it is missing or older than its
    sources."""
    os.makedirs(OUT_DIR, exist_ok=True)
    hdr = os.path.join(HERE, "pf_oracle.h")
    lib = LIB_OMP if openmp else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC"]
    cmd += ["-fopenmp"] if openmp else ["-Wno-unknown-pragmas"]
    cmd += ["-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
