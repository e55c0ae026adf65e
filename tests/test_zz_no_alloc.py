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


def test_totals_noalloc_capped_blocks_field_limit_and_nan(env):
    torch, pf, L = env
    rng = np.random.default_rng(7)
    # 2.2 M cells: more than 512 blocks of 4096 cells, so the block count is
    # capped and every block reduces a larger chunk
    V = 2_200_001
    u = rng.random((2, V)) - 0.25
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    maxes = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(2):                                  # two calls in a row
        assert L.pf_totals_noalloc(ud.data_ptr(), 2, V, 0.5, sums.data_ptr(), maxes.data_ptr(), None) == pf.PF_OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(sums.cpu().numpy(), 0.5 * u.sum(axis=1), rtol=1e-12)
        np.testing.assert_array_equal(maxes.cpu().numpy(), u.max(axis=1))
    # the largest field count, the last scratch rows in use
    u = rng.random((130, 999)) * 2.0 - 1.0
    u[129, 17] = -np.inf                               # a maximum below -1e300 is still exact
    u[129, :17] = -np.inf
    u[129, 18:] = -np.inf
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    sums = torch.zeros(130, dtype=torch.float64, device="cuda")
    maxes = torch.zeros(130, dtype=torch.float64, device="cuda")
    assert L.pf_totals_noalloc(ud.data_ptr(), 130, 999, 1.0, sums.data_ptr(), maxes.data_ptr(), None) == pf.PF_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(sums.cpu().numpy()[:129], u[:129].sum(axis=1), rtol=1e-12)
    np.testing.assert_array_equal(maxes.cpu().numpy(), u.max(axis=1))
    # a NaN makes that field's sum and maximum NaN, the others are unaffected
    u = rng.random((3, 5000))
    u[1, 4321] = np.nan
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    maxes = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert L.pf_totals_noalloc(ud.data_ptr(), 3, 5000, 1.0, sums.data_ptr(), maxes.data_ptr(), None) == pf.PF_OK
    torch.cuda.synchronize()
    s, m = sums.cpu().numpy(), maxes.cpu().numpy()
    assert np.isnan(s[1]) and np.isnan(m[1])
    np.testing.assert_allclose(s[[0, 2]], u[[0, 2]].sum(axis=1), rtol=1e-12)
    np.testing.assert_array_equal(m[[0, 2]], u[[0, 2]].max(axis=1))
