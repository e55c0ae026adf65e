"""CPU-only checks of the boundary: the library builds, loads without a GPU and
exports every entry point that include/pf.h declares; the product package
does not depend on the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pf\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2601_16522_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "pf_create" in names and "pf_step" in names and "pf_get_state" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_2601_16522_gb300 import pf
    lib = pf.lib()
    assert lib.pf_strerror(0) == b"ok"
    assert b"invalid" in lib.pf_strerror(1)


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2601_16522_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
                assert "pf_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            for m in re.findall(r"^\s*(?:from|import)\s+(paper_2601_16522_gb300[\w.]*)", txt, re.M):
                assert m == "paper_2601_16522_gb300.inputs", (f, m)
            assert "pf_kernels" not in txt and "include/pf.h" not in txt, f


def test_instantiation_units_match_their_generator():
    # the committed pf_stage_*.cu files are what csrc/gen_units.py writes
    import importlib.util
    path = os.path.join(ROOT, "paper_2601_16522_gb300", "csrc", "gen_units.py")
    spec = importlib.util.spec_from_file_location("gen_units", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    for name, text in gen.render().items():
        with open(os.path.join(os.path.dirname(path), name)) as f:
            assert f.read() == text, name


def test_binding_structs_match_the_header(tmp_path):
    # The ctypes mirrors of pf_params, pf_tol, pf_step_opts and pf_stats must
    # have the C layout: compile a probe against include/pf.h and compare the
    # size and every field offset.
    import shutil
    import subprocess
    from paper_2601_16522_gb300 import pf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pf_params": pf.pf_params, "pf_tol": pf.pf_tol, "pf_step_opts": pf.pf_step_opts,
               "pf_stats": pf.pf_stats, "pf_controller": pf.pf_controller}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pf.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_argument_checks_without_gpu():
    # Entry points reject bad arguments before any device work, so these run
    # without a GPU: a null handle, a null output, a poll limit out of range.
    from paper_2601_16522_gb300 import pf
    L = pf.lib()
    ctl = pf.pf_controller()
    assert L.pf_get_controller(None, ctypes.byref(ctl)) == 1
    assert L.pf_set_controller(None, ctypes.byref(ctl)) == 1
    assert L.pf_selftest_wait(None, 0) == 1
    assert L.pf_selftest_wait(None, (1 << 22) + 1) == 1
    d = ctypes.c_double()
    assert L.pf_dt_e(None, ctypes.byref(d)) == 1
    assert L.pf_energy(None, ctypes.byref(d)) == 1
    assert L.pf_destroy(None) == 0


def test_create_rejects_degenerate_and_invalid_problems():
    # pf_create validates every parameter before it touches a device, so the
    # degenerate and invalid cases run without a GPU; each must be PF_EINVAL.
    import numpy as np
    from paper_2601_16522_gb300 import inputs as I
    from paper_2601_16522_gb300 import pf
    L = pf.lib()
    prob, _ = I.multiphase_blobs(8, 6, 1, 3, seed=1, has_conc=1, n_alpha=1)
    cases = {
        "empty grid": dict(nx=0),
        "2D with nz > 1": dict(nz=2),
        "dx = 0": dict(dx=0.0),
        "W < 0": dict(W=-1.0),
        "one phase": dict(n_phases=1, phase_type=np.array([0], np.int32), gamma=np.zeros((1, 1)),
                          mobility=np.zeros((1, 1))),
        "more than 128 fields": dict(n_phases=130, phase_type=np.ones(130, np.int32),
                                     gamma=I.uniform_pairs(130, 1.0), mobility=I.uniform_pairs(130, 1.0)),
        "phase type 2": dict(phase_type=np.array([0, 2, 1], np.int32)),
        "k = 0": dict(k=(0.0, 1.0)),
        "periodic opposite Neumann": dict(bc_phi=(0, 1, 0, 0, 0, 0)),
        "Dirichlet phase field": dict(bc_phi=(2, 2, 0, 0, 0, 0), bc_c=(2, 2, 0, 0, 0, 0)),
        "c periodic against phi Neumann": dict(bc_phi=(1, 1, 0, 0, 0, 0), bc_c=(0, 0, 0, 0, 0, 0)),
        "non-finite c_ref": dict(c_ref=float("inf")),
    }
    for name, kw in cases.items():
        p, keep = pf.make_params(prob.with_(**kw), precision=32)
        h = ctypes.c_void_p()
        assert L.pf_create(ctypes.byref(p), None, ctypes.byref(h)) == 1, name
        assert not h.value, name
    p, keep = pf.make_params(prob, precision=16)
    assert L.pf_create(ctypes.byref(p), None, ctypes.byref(ctypes.c_void_p())) == 1
    p, keep = pf.make_params(prob, precision=64)
    p.dim = 1
    assert L.pf_create(ctypes.byref(p), None, ctypes.byref(ctypes.c_void_p())) == 1
    assert L.pf_create(None, None, ctypes.byref(ctypes.c_void_p())) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # No CPU fallback: without the compiled library every entry point raises
    # ImportError instead of computing anything another way.
    from paper_2601_16522_gb300 import inputs as I
    from paper_2601_16522_gb300 import pf
    monkeypatch.setattr(pf, "_LIB", None)
    monkeypatch.setattr(pf, "LIB_PATH", str(tmp_path / "absent" / "libpf.so"))
    prob, _ = I.circle(16, 4.0)
    with pytest.raises(ImportError):
        pf.Simulation(prob, precision=64)
    with pytest.raises(ImportError):
        pf.footprint(prob)
    with pytest.raises(ImportError):
        pf.selftest_wait(16)


def test_plain_c_caller_links_and_runs(tmp_path):
    # The boundary from C itself: a C99 program includes include/pf.h, links
    # libpf.so and calls the entry points that need no device (status text,
    # parameter validation, argument checks).
    import shutil
    import subprocess
    from paper_2601_16522_gb300 import pf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pf.lib()                                                  # built
    libdir = os.path.dirname(pf.LIB_PATH)
    src = tmp_path / "caller.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "pf.h"
int main(void) {
    int ptype[2] = {0, 0};
    double gam[4] = {0, 1, 1, 0}, mob[4] = {0, 1, 1, 0};
    pf_params p;
    memset(&p, 0, sizeof p);
    p.dim = 2; p.nx = 0; p.ny = 8; p.nz = 1; p.dx = 1.0; p.n_phases = 2;   /* empty grid */
    p.phase_type = ptype; p.gamma = gam; p.mobility = mob; p.W = 2.0; p.precision = 64;
    struct pf_handle *h = 0;
    int s1 = pf_create(&p, 0, &h);
    pf_controller c;
    int s2 = pf_get_controller(0, &c);
    int s3 = pf_selftest_wait(0, 0);
    int s4 = pf_destroy(0);
    printf("%d %d %d %d %d %s\n", s1, h == 0, s2, s3, s4, pf_strerror(PF_EINVAL));
    return 0;
}
""")
    exe = tmp_path / "caller"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lpf", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[:5] == ["1", "1", "1", "1", "0"]
    assert "invalid" in " ".join(out[5:])
