"""pf_totals_noalloc: the allocation-free totals entry point.

Some callers cannot allocate device memory where they need the totals
(cudaMalloc/cudaFree may synchronise the device; an external allocator may
own all memory).  pf_totals_noalloc uses a fixed scratch array inside the
library instead; here it must agree with pf_reduce (which allocates its
scratch at pf_create) on two calls in a row with different states.
This file is collected last so that a failure here does not stop the run
before the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16522_gb300 import build
    build.build()
    from paper_2601_16522_gb300 import pf
    L = pf.lib()
    L.pf_totals_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_longlong, C.c_double, C.c_void_p, C.c_void_p,
                                    C.c_void_p]
    L.pf_totals_noalloc.restype = C.c_int
    return torch, pf, L


def test_totals_noalloc_matches_pf_reduce(env):
    torch, pf, L = env
    for seed, shape in ((31, (20, 18, 16)), (32, (37, 11, 9))):     # two calls in a row
        prob, u = I.multiphase_blobs(*shape, 6, seed=seed, has_conc=1, n_alpha=2)
        N, NF, V = prob.n_phases, prob.nfields, prob.V
        dv = prob.dx ** prob.dim
        with pf.Simulation(prob, precision=64) as sim:
            sim.set_state(u)
            mass, vol, alive = sim.reduce()
        ud = torch.tensor(u, dtype=torch.float64, device="cuda")
        sums = torch.full((NF,), -1.0, dtype=torch.float64, device="cuda")
        maxes = torch.full((NF,), -1.0, dtype=torch.float64, device="cuda")
        st = L.pf_totals_noalloc(ud.data_ptr(), NF, V, dv, sums.data_ptr(), maxes.data_ptr(), None)
        torch.cuda.synchronize()
        assert st == pf.PF_OK
        s = sums.cpu().numpy()
        m = maxes.cpu().numpy()
        np.testing.assert_allclose(s[:N], vol, rtol=1e-12)
        assert s[N] == pytest.approx(mass, rel=1e-12)
        assert int((m[:N] >= 0.5).sum()) == alive
        np.testing.assert_array_equal(m, u.max(axis=1))


def test_totals_noalloc_rejects_oversize(env):
    torch, pf, L = env
    ud = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(200, dtype=torch.float64, device="cuda")
    st = L.pf_totals_noalloc(ud.data_ptr(), 131, 8, 1.0, out.data_ptr(), None, None)
    assert st == pf.PF_EINVAL
    st = L.pf_totals_noalloc(ud.data_ptr(), 4, 8, 1.0, None, None, None)
    assert st == pf.PF_EINVAL
