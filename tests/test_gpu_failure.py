"""Failure detection without a GPU fault: a bounded device wait that runs out
reports PF_ETIMEOUT to the host and leaves the context usable.

pf_selftest_wait makes one thread wait on a shared-memory mbarrier that no
thread arrives on, with the poll loop the TMA-staged kernels use (their
waits give up after 2^22 polls and raise the same flag)."""
import time

import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

PF_EINVAL, PF_ETIMEOUT = 1, 4


def test_bounded_wait_times_out_and_context_survives(pf):
    import torch
    t0 = time.perf_counter()
    assert pf.selftest_wait(1 << 16) == PF_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert pf.selftest_wait(1 << 10, stream=torch.cuda.Stream()) == PF_ETIMEOUT
    assert pf.selftest_wait(0) == PF_EINVAL and pf.selftest_wait(1 << 23) == PF_EINVAL
    # the context is intact: a normal run afterwards is well defined
    prob, u = I.circle(32, 9.0, W=2.5)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        st = sim.step(pf.FEULER, 10 * 0.9 * sim.dt_e(), dt_mult=0.9)
        ug, _ = sim.get_state()
    assert st["rhs_evals"] == 10 and np.isfinite(ug).all()
    assert np.abs(ug.sum(0) - 1.0).max() < 1e-12


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("field,integ,kw", [
    ("phase", I.FEULER, dict(dt_mult=0.9)),
    ("phase", I.RKL2, dict(tol=(1e-4, 1e-3, 1e-4, 1e-4))),
    ("conc", I.RKL2, dict(tol=(1e-4, 1e-3, 1e-4, 1e-4))),
], ids=["phase-fe", "phase-rkl2", "conc-rkl2"])
def test_non_finite_state_is_reported(pf, field, integ, kw, prec):
    # A non-finite value makes the simplex sum of its cell fail (phases: the
    # projection checks sum > 0, false for NaN) or the error norm non-finite
    # (adaptive steps: every concentration entry enters the norm); either way
    # the step ends with PF_EUNSTABLE (the contract of pf_step), and the
    # handle still answers.
    prob, good = I.multiphase_blobs(17, 13, 1, 4, seed=3, has_conc=1, n_alpha=1)
    u = good.copy()
    if field == "phase":
        u[1, 100] = np.nan
    else:
        u[prob.n_phases, 100] = np.nan
    with pf.Simulation(prob, precision=prec) as sim:
        sim.set_state(u)
        with pytest.raises(pf.PfError) as e:
            sim.step(integ, 5 * sim.dt_e(), **kw)
        assert e.value.status == 3                     # PF_EUNSTABLE
        sim.set_state(good)
        st = sim.step(integ, 5 * sim.dt_e(), **kw)
        assert st["t"] == pytest.approx(5 * sim.dt_e())


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "launched"])
@pytest.mark.parametrize("integ,mult", [(I.FEULER, 3.0), (I.SSP2, 12.0)], ids=["fe", "ssp2"])
def test_fixed_steps_end_at_the_last_good_step(pf, integ, mult, graph, prec):
    # Fixed steps far beyond the stable step (3x for forward Euler, 3x the
    # (s-1) dt_e limit of SSP(5)2) make the concentration grow without bound
    # until a pass flags a non-finite value or simplex sum.  pf_step must then
    # return PF_EUNSTABLE with the state and time of the last step that
    # completed cleanly (every later pass does nothing), whether the steps
    # were replayed from a CUDA graph or launched one by one.
    import torch
    prob, u = I.multiphase_blobs(17, 13, 1, 4, seed=3, has_conc=1, n_alpha=1)
    flags = 0 if graph else pf.Simulation.STEP_NO_GRAPH
    with pf.Simulation(prob, precision=prec, stream=torch.cuda.Stream()) as sim:
        sim.set_state(u)
        dt = mult * sim.dt_e()
        t_end = 2000 * dt
        with pytest.raises(pf.PfError) as e:
            sim.step(integ, t_end, dt_mult=mult, ssp_stages=5, flags=flags)
        assert e.value.status == pf.PF_EUNSTABLE
        ug, t = sim.get_state()
    k = int(round(t / dt))
    assert 1 <= k < 2000 and t == k * dt
    assert np.isfinite(ug).all()
    assert np.abs(ug[:prob.n_phases].sum(0) - 1.0).max() < (1e-12 if prec == 64 else 1e-5)
    with pf.Simulation(prob, precision=prec, stream=torch.cuda.Stream()) as sim:
        sim.set_state(u)
        # the same k steps (every one of size dt) end cleanly at the same state
        st = sim.step(integ, t_end, dt_mult=mult, ssp_stages=5, max_attempts=k, flags=flags)
        assert st["steps_accepted"] == k and st["t"] == t
        u2, _ = sim.get_state()
        np.testing.assert_array_equal(u2, ug)
        # and the next step fails, leaving that state and time
        with pytest.raises(pf.PfError) as e:
            sim.step(integ, t_end, dt_mult=mult, ssp_stages=5, flags=flags)
        assert e.value.status == pf.PF_EUNSTABLE
        u3, t3 = sim.get_state()
        assert t3 == t
        np.testing.assert_array_equal(u3, ug)
