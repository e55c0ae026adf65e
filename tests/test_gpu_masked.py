"""Masked storage (PF_OPT_MASKED): the occupancy-masked FP32 passes against
the dense FP32 passes and the FP64 oracle.

A phase outside a cell's occupancy union has an exactly zero RHS and stage
value, so skipping it changes nothing but the sign of some zeros: the masked
results equal those of the dense one-cell kernels (PF_OPT_ONE_CELL, the same
arithmetic) value for value (np.array_equal treats -0 and +0 as equal).  The dense FP32 path is itself tested against the oracle
in test_gpu_parity.py; here the masked path is also compared with the
oracle directly on one RKL2 step of a 32-grain 3D state.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import CASES, pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

ELIGIBLE = [c for c in CASES if c[0] != "blobs3d_N70"]
N70 = [c for c in CASES if c[0] == "blobs3d_N70"][0]
TOL = (1e-4, 1e-3, 1e-4, 1e-3)
ONE = 4          # PF_OPT_ONE_CELL: the dense kernels the masked ones are bit-equal to


def _run(pf, prob, u, opts, integ, nsteps_dte, **kw):
    with pf.Simulation(prob, precision=32, options=opts) as sim:
        sim.set_state(u)
        st = sim.step(integ, nsteps_dte * sim.dt_e(), **kw)
        out, t = sim.get_state()
    return out, st


@pytest.mark.parametrize("integ,kw", [(ref.FEULER, dict(dt_mult=0.9)), (ref.SSP2, dict(dt_mult=2.0)),
                                      (ref.RKL1, dict(dt_mult=6.0)), (ref.RKL2, dict(dt_mult=12.0)),
                                      (ref.SSP104, dict(dt_mult=2.0))],
                         ids=["fe", "ssp2", "rkl1", "rkl2", "ssp104"])
@pytest.mark.parametrize("name,prob,u", ELIGIBLE, ids=[c[0] for c in ELIGIBLE])
def test_masked_fixed_steps_equal_dense(pf, name, prob, u, integ, kw):
    n = 10 if integ != ref.FEULER else 6
    dense, st_d = _run(pf, prob, u, ONE, integ, n, **kw)
    masked, st_m = _run(pf, prob, u, pf.Simulation.OPT_MASKED, integ, n, **kw)
    assert st_d["rhs_evals"] == st_m["rhs_evals"]
    assert np.array_equal(masked, dense), np.abs(masked - dense).max()


def test_masked_three_words_fe_equal_dense(pf):
    # 70 phases: three occupancy words per cell; one forward Euler step (the
    # 70-phase blob state exceeds the 12-phase list capacity after that)
    name, prob, u = N70
    dense, st_d = _run(pf, prob, u, ONE, ref.FEULER, 0.9, dt_mult=0.9)
    masked, st_m = _run(pf, prob, u, pf.Simulation.OPT_MASKED, ref.FEULER, 0.9, dt_mult=0.9)
    assert np.array_equal(masked, dense), np.abs(masked - dense).max()


@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2, ref.SSP104], ids=["rkl1", "rkl2", "ssp104"])
@pytest.mark.parametrize("name,prob,u", [ELIGIBLE[1], ELIGIBLE[3], ELIGIBLE[-1]],
                         ids=[ELIGIBLE[1][0], ELIGIBLE[3][0], ELIGIBLE[-1][0]])
def test_masked_adaptive_equal_dense(pf, name, prob, u, integ):
    dense, st_d = _run(pf, prob, u, ONE, integ, 40, tol=TOL)
    masked, st_m = _run(pf, prob, u, pf.Simulation.OPT_MASKED, integ, 40, tol=TOL)
    for k in ("rhs_evals", "steps_accepted", "steps_rejected"):
        assert st_d[k] == st_m[k], k
    assert np.array_equal(masked, dense), np.abs(masked - dense).max()


def test_masked_grains_rkl2_vs_oracle(pf):
    # 48^3, 32 grains: one RKL2 step of 9 dt_e in masked storage, replayed
    # by the FP64 oracle on the FP32-rounded initial state
    prob, u = I.grains_device(n=48, n_grains=32, min_dist=9.0, seed=5, dim=3, dx=1.0, W_cells=2.5, M=1.0,
                              device="cuda")
    u = u.cpu().numpy()
    with pf.Simulation(prob, precision=32, options=pf.Simulation.OPT_MASKED) as sim:
        sim.set_state(u)
        u32, _ = sim.get_state()
        dt = 9.0 * sim.dt_e()
        st = sim.step(pf.RKL2, dt, dt_mult=9.0, trace_cap=4)
        out, _ = sim.get_state()
    with pf.Simulation(prob, precision=32, options=ONE) as sim:
        sim.set_state(u)
        sim.step(pf.RKL2, dt, dt_mult=9.0)
        dense, _ = sim.get_state()
    assert np.array_equal(out, dense)
    tr = st["trace"]
    assert len(tr["dt"]) == 1
    o = ref.Oracle(prob)
    un, _, _, _ = o.step(ref.RKL2, tr["dt"][0], int(tr["s"][0]), u32)
    scale = np.abs(un).max()
    assert np.abs(out - un).max() <= 2e-5 * scale


def test_masked_grains_ssp104_vs_oracle(pf):
    # 48^3, 32 grains, K = 1: one adaptive SSP(10)4 attempt in masked storage
    # (the z accumulator, the q2 combination and the embedded error in the
    # masked passes) equals the dense one-cell passes, and the FP64 oracle's
    # step and embedded error norm from the same FP32-rounded state
    prob, u = I.sintering_device(n=48, n_grains=24, seed=3, device="cuda")
    u = u.cpu().numpy()
    tol = (1e-4, 1e-3, 1e-4, 1e-3)
    res = []
    for opts in (pf.Simulation.OPT_MASKED, ONE):
        with pf.Simulation(prob, precision=32, options=opts) as sim:
            sim.set_state(u)
            u32, _ = sim.get_state()
            dt0 = 3.0 * sim.dt_e()
            st = sim.step(pf.SSP104, 1e30, tol=tol, dt0=dt0, max_attempts=1, trace_cap=2)
            out, _ = sim.get_state()
        res.append((st, out, u32))
    (st_m, out_m, u32), (st_d, out_d, _) = res
    assert np.array_equal(out_m, out_d)
    assert st_m["trace"]["err"][0] == st_d["trace"]["err"][0]
    o = ref.Oracle(prob)
    un, err, nd = o.step_error(ref.SSP104, st_m["trace"]["dt"][0], 10, u32, tol)
    N = prob.n_phases
    scale = np.abs(un[:N]).max()
    assert np.abs(out_m[:N] - un[:N]).max() <= 2e-5 * scale
    # e = u - z of FP32 values after ten stages: a few 1e-7 absolute per entry
    # against weights of about a_phi = 1e-3
    assert abs(st_m["trace"]["err"][0] - err) <= 2e-2 * err + 1e-3


def test_masked_graph_replay_equals_launches(pf):
    name, prob, u = ELIGIBLE[3]
    outs = []
    for flags in (0, pf.Simulation.STEP_NO_GRAPH):
        with pf.Simulation(prob, precision=32, options=pf.Simulation.OPT_MASKED) as sim:
            sim.set_state(u)
            sim.step(ref.RKL2, 40 * sim.dt_e(), dt_mult=4.0, flags=flags)
            outs.append(sim.get_state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_masked_eligibility_and_footprint(pf):
    name, prob, u = ELIGIBLE[0]
    with pytest.raises(RuntimeError):
        pf.Simulation(prob, precision=64, options=pf.Simulation.OPT_MASKED)
    for name, prob, u in (ELIGIBLE[0], N70):
        d = pf.footprint(prob, 32)
        m = pf.footprint(prob, 32, options=pf.Simulation.OPT_MASKED)
        Vs = (prob.V + 63) // 64 * 64
        assert m - d == 5 * ((prob.n_phases + 31) // 32) * Vs * 4
