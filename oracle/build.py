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


def build(force=False):
    """Compile ``liboracle.so`` if it is missing or older than its sources."""
    os.makedirs(OUT_DIR, exist_ok=True)
    hdr = os.path.join(HERE, "pf_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
