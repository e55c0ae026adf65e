"""The mobility-weighted projection (PF_OPT_MOBILITY_SIMPLEX, a reading of
the mobility-based simplex Sec. 3.1 cites for the particle cases of
Sec. 5.3) on the GPU against the oracle's or_project_cell_mobility: FP64
within 1e-12 of the oracle's step, FP32 within a few FP32 roundings; its
incompatible options are refused."""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import REL64, pf, relerr  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _cases():
    c = []
    prob, u = I.multiphase_blobs(17, 13, 1, 5, seed=3, has_conc=1, n_alpha=2)
    c.append(("blobs2d_K1", prob.with_(simplex=1), u))
    prob, u = I.multiphase_blobs(10, 9, 7, 6, seed=6, has_conc=0, bc_phi=(1, 1, 0, 0, 1, 1))
    c.append(("blobs3d_neumann", prob.with_(simplex=1), u))
    return c


CASES = _cases()
STEPS = [(ref.FEULER, 1, 0.9), (ref.SSP2, 5, 2.0), (ref.SSP104, 10, 3.0), (ref.RKL1, 0, 30.0), (ref.RKL2, 0, 60.0)]


@pytest.mark.parametrize("integ,s,mult", STEPS, ids=["fe", "ssp2", "ssp104", "rkl1", "rkl2"])
@pytest.mark.parametrize("name,prob,u", CASES, ids=[c[0] for c in CASES])
def test_single_step_fp64_and_fp32(pf, name, prob, u, integ, s, mult):
    o = ref.Oracle(prob)
    N, K = prob.n_phases, prob.has_conc
    for prec in (64, 32):
        with pf.Simulation(prob, precision=prec) as sim:
            sim.set_state(u)
            u0, _ = sim.get_state()
            dt = mult * sim.dt_e()
            st = sim.step(integ, dt, dt_mult=mult, ssp_stages=max(s, 2), trace_cap=2)
            out, t = sim.get_state()
        s_used = int(st["trace"]["s"][0])
        un, _, _, _ = o.step(integ, dt, s_used, u0)
        if prec == 64:
            assert relerr(out, un, N, K) <= REL64
        else:
            assert np.abs(out[:N] - un[:N]).max() <= 2e-5 * max(s_used, 1) ** 0.5


def test_projection_acts_and_differs_from_the_standard_one(pf):
    # the RKL2 step at 60 dt_e moves interfaces enough that the projection
    # acts in many cells; the two projections give different states
    name, prob, u = CASES[0]
    outs = []
    for p in (prob, prob.with_(simplex=0)):
        with pf.Simulation(p, precision=64) as sim:
            sim.set_state(u)
            sim.step(ref.RKL2, 60 * sim.dt_e(), dt_mult=60.0)
            outs.append(sim.get_state()[0])
    assert np.abs(outs[0] - outs[1]).max() > 1e-6
    N = prob.n_phases
    assert outs[0][:N].min() >= 0.0
    np.testing.assert_allclose(outs[0][:N].sum(axis=0), 1.0, atol=1e-13)


def test_immobile_particles_with_the_mobility_simplex(pf):
    # Sec. 5.3 particles (radius 6, fraction 0.15) with the immobile
    # parameters, adaptive RKL2 in FP64 for a few attempts: every attempt is
    # the oracle's step from the same state
    prob, ud = I.zener_device(n=40, n_grains=10, device="cuda")
    prob = prob.with_(simplex=1)
    u = ud.cpu().numpy()
    o = ref.Oracle(prob)
    tol = (1e-4, 1e-2, 1e-4, 1e-3)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        st = sim.step(ref.RKL2, 1e30, tol=tol, dt0=30 * sim.dt_e(), max_attempts=1, trace_cap=2)
        out, _ = sim.get_state()
    tr = st["trace"]
    un, err, _ = o.step_error(ref.RKL2, tr["dt"][0], int(tr["s"][0]), u, tol)
    if tr["acc"][0]:
        assert relerr(out, un, prob.n_phases, 1) <= REL64
    # the norm's entry count can move by one between rounding orders
    assert abs(tr["err"][0] - err) <= 2e-2 * err


def test_incompatible_options_are_refused(pf):
    name, prob, u = CASES[0]
    with pytest.raises(RuntimeError):
        pf.Simulation(prob, precision=32, options=pf.Simulation.OPT_MASKED)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        with pytest.raises(RuntimeError):
            sim.step(ref.RKL2, 20 * sim.dt_e(), tol=(1e-4,) * 4, flags=pf.Simulation.STEP_REUSE_RHS)
