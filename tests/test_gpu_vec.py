"""The two-cell FP32 kernels (default for dense FP32 storage with nx even)
against the one-cell kernels (PF_OPT_ONE_CELL) and the FP64 oracle.

Both evaluate the same stage arithmetic in FP32 (combination, projection,
first-stage fix, error terms); the two-cell kernel forms the Laplacian and
the concentration sums in another order, so results agree to FP32 rounding,
not bit for bit.  Shapes cover ragged tiles (nx not a multiple of 64, ny not
a multiple of 4), every boundary kind, K = 0 and 1, 2D and 3D, N = 2 to 70
(rolled phase loop beyond 64: the second rewrite mask), and cells with more
nontrivial phases than the 8-entry list (the wide path)."""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import pf, relerr  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

TOL = (1e-4, 1e-3, 1e-4, 1e-4)


def _cases():
    c = []
    prob, u = I.circle(48, 12.0, W=2.5, ny=38)
    c.append(("circle48x38", prob, u))
    prob, u = I.multiphase_blobs(70, 22, 1, 5, seed=3, has_conc=1, n_alpha=2)
    c.append(("blobs2d_K1", prob, u))
    prob, u = I.multiphase_blobs(66, 14, 1, 4, seed=4, has_conc=1, n_alpha=1,
                                 bc_phi=(1, 1, 0, 0, 0, 0), bc_c=(2, 1, 0, 0, 0, 0),
                                 c_dirichlet=(0.7, 0.0, 0, 0, 0, 0))
    c.append(("blobs2d_bcx", prob, u))
    prob, u = I.multiphase_blobs(20, 18, 9, 6, seed=6, has_conc=1, n_alpha=1,
                                 bc_phi=(0, 0, 1, 1, 1, 1), bc_c=(0, 0, 2, 1, 2, 2),
                                 c_dirichlet=(0, 0, 0.6, 0, 0.3, 0.5))
    c.append(("blobs3d_bcyz", prob, u))
    prob, u = I.multiphase_blobs(32, 30, 28, 33, seed=8, has_conc=1, n_alpha=3, min_dist=8.0)
    c.append(("blobs3d_N33", prob, u))
    prob, u = I.multiphase_blobs(30, 28, 26, 70, seed=9, has_conc=0, min_dist=5.0)
    c.append(("blobs3d_N70", prob, u))
    prob, u = I.multiphase_blobs(10, 9, 8, 40, seed=9, has_conc=0, min_dist=1.5)
    c.append(("crowded_N40", prob, u))
    return c


CASES = _cases()
STEPS = [(ref.FEULER, 1, 0.5), (ref.SSP2, 5, 2.0), (ref.RKL1, 0, 12.0), (ref.RKL2, 0, 25.0)]


@pytest.mark.parametrize("integ,s,mult", STEPS, ids=["fe", "ssp2", "rkl1", "rkl2"])
@pytest.mark.parametrize("name,prob,u", CASES, ids=[c[0] for c in CASES])
def test_two_cell_step_matches_one_cell_and_oracle(pf, name, prob, u, integ, s, mult):
    u = u.astype(np.float32).astype(np.float64)
    assert prob.nx % 2 == 0
    o = ref.Oracle(prob)
    dte = o.dt_e()
    dt = mult * dte
    if integ in (ref.RKL1, ref.RKL2):
        s = ref.sts_stages(integ, dt, dte)
    ref64, _, _, _ = o.step(integ, dt, s, u)
    out = []
    for opt in (0, pf.Simulation.OPT_ONE_CELL):
        with pf.Simulation(prob, precision=32, options=opt) as sim:
            sim.set_state(u)
            st = sim.step(integ, dt, dt_mult=mult, ssp_stages=s if integ == ref.SSP2 else 5)
            out.append(sim.get_state()[0])
            assert st["rhs_evals"] == (s if integ != ref.FEULER else 1)
    two, one = out
    N, K = prob.n_phases, prob.has_conc
    # FP32 against FP32 (different summation orders) and against FP64
    tol = 2e-5 if integ in (ref.FEULER, ref.SSP2) else 2e-4
    assert relerr(two, one, N, K) <= tol
    assert relerr(two, ref64, N, K) <= 5 * tol
    assert np.abs(two[:N].sum(0) - 1.0).max() < 1e-5


@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2], ids=["rkl1", "rkl2"])
@pytest.mark.parametrize("name,prob,u", [CASES[1], CASES[3], CASES[5]], ids=["blobs2d_K1", "blobs3d_bcyz", "N70"])
def test_two_cell_error_sweep_matches_the_oracle(pf, name, prob, u, integ):
    # the first attempt's error norm (Sec. 3.3) from a common FP32-rounded
    # state: the oracle evaluates it in FP64 on the same input
    u = u.astype(np.float32).astype(np.float64)
    o = ref.Oracle(prob)
    dte = o.dt_e()
    dt0 = 8.0 * dte
    with pf.Simulation(prob, precision=32) as sim:
        sim.set_state(u)
        st = sim.step(integ, 1e9, tol=TOL, dt0=dt0, max_attempts=1, trace_cap=4)
        tr = st["trace"]
    s = tr["s"][0]
    _, e_ref, _ = o.step_error(integ, dt0, s, u, TOL)
    assert tr["err"][0] == pytest.approx(e_ref, rel=2e-3)


def test_two_cell_crowded_cells_take_the_wide_path(pf):
    # more than 8 nontrivial phases in a cell: past the two-cell list
    name, prob, u = CASES[6]
    u = u.astype(np.float32).astype(np.float64)
    o = ref.Oracle(prob)
    _, nz = o.rhs(u)
    assert (nz > 8).sum() > 20 and nz.max() > 12
    dte = o.dt_e()
    fe_ref, _, _, _ = o.step(ref.FEULER, 0.5 * dte, 1, u)
    with pf.Simulation(prob, precision=32) as sim:
        sim.set_state(u)
        sim.step(ref.FEULER, 0.5 * dte, dt_mult=0.5)
        assert relerr(sim.get_state()[0], fe_ref, prob.n_phases, 0) <= 2e-5


def test_adaptive_rkl2_two_cell_and_one_cell_agree(pf):
    # adaptive RKL2 over a few steps: the same attempts, states within FP32 rounding
    prob, u = I.multiphase_blobs(48, 36, 1, 5, seed=3, has_conc=1, n_alpha=2)
    runs = []
    for opt in (0, pf.Simulation.OPT_ONE_CELL):
        with pf.Simulation(prob, precision=32, options=opt) as sim:
            sim.set_state(u)
            st = sim.step(ref.RKL2, 40 * sim.dt_e(), tol=TOL, trace_cap=1000)
            runs.append((st, sim.get_state()[0]))
    (sa, ua), (sb, ub) = runs
    np.testing.assert_array_equal(sa["trace"]["s"], sb["trace"]["s"])
    np.testing.assert_array_equal(sa["trace"]["acc"], sb["trace"]["acc"])
    np.testing.assert_allclose(sa["trace"]["err"], sb["trace"]["err"], rtol=1e-3)
    assert relerr(ua, ub, prob.n_phases, prob.has_conc) <= 1e-4


def test_autotune_reports_every_applicable_variant(pf):
    prob, u = I.multiphase_blobs(64, 32, 16, 6, seed=1, has_conc=0)
    with pf.Simulation(prob, precision=32) as sim:
        sim.set_state(u)
        choice, ms = sim.autotune()
        assert set(ms) == {0, 1, 2} and choice == min(ms, key=ms.get)
        st = sim.step(ref.RKL2, 10 * sim.dt_e(), tol=TOL)
        assert st["t"] == pytest.approx(10 * sim.dt_e())
    prob2, u2 = I.multiphase_blobs(33, 20, 1, 4, seed=1)          # odd nx: no two-cell kernel
    with pf.Simulation(prob2, precision=32) as sim:
        sim.set_state(u2)
        choice, ms = sim.autotune()
        assert set(ms) == {1} and choice == 1
