"""Build libpf.so (the sm_103a engine) in-tree with nvcc.

The translation units compile in parallel: the FP64 stage pass (built with
``--fmad=false`` so its arithmetic is exactly the written sequence of
IEEE operations), the FP32 stage passes for K = 0 and K = 1 in dense and
masked storage (FMA contraction on), the dispatch, the allocation-free totals
and the host engine.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]
UNITS = [
    ("pf_stage_f64.cu", ["--fmad=false"]),
    ("pf_stage_f32k0.cu", ["--fmad=true"]),
    ("pf_stage_f32k1.cu", ["--fmad=true"]),
    ("pf_stage_m32k0.cu", ["--fmad=true"]),
    ("pf_stage_m32k1.cu", ["--fmad=true"]),
    ("pf_stage_v32k0.cu", ["--fmad=true"]),
    ("pf_stage_v32k1.cu", ["--fmad=true"]),
    ("pf_stage_s32k0.cu", ["--fmad=true"]),
    ("pf_stage_s32k1.cu", ["--fmad=true"]),
    ("pf_dispatch.cu", ["--fmad=false"]),
    ("pf_noalloc.cu", ["--fmad=false"]),
    ("pf_engine.cu", ["--fmad=false"]),
]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "pf.h")]


def build(force=False, verbose=False, ptxas_info=False):
    """Compile every CUDA unit for sm_103a and link ``libpf.so`` (no-op if up to date)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    extra += os.environ.get("PF_NVCC_EXTRA", "").split()

    def compile_unit(unit):
        name, flags = unit
        obj = os.path.join(OUT_DIR, name.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + COMMON + flags + extra + ["-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, r.stdout, r.stderr))
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
