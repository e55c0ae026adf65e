"""Checkpoint and resume of an adaptive run: pf_get_state + pf_get_controller
on one handle, pf_set_state + pf_set_controller on another; the continued
run must take the same steps and end in the same state as the run that was
never interrupted (the kernels and the FP64 reductions are deterministic)."""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

TOL = (1e-4, 1e-3, 1e-4, 1e-4)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("integ", [ref.RKL2, ref.SSP104], ids=["rkl2", "ssp104"])
def test_resumed_run_equals_uninterrupted(pf, integ, prec):
    prob, u = I.multiphase_blobs(17, 13, 9, 5, seed=3, has_conc=1, n_alpha=2)
    with pf.Simulation(prob, precision=prec) as a:
        a.set_state(u)
        t1, t2 = 20 * a.dt_e(), 60 * a.dt_e()
        a.step(integ, t1, tol=TOL)
        u1, tt = a.get_state()
        ctrl = a.get_controller()
        s2 = a.step(integ, t2, tol=TOL, trace_cap=1000)
        ua, _ = a.get_state()
    assert tt == t1 and ctrl["nhist"] >= 1 and ctrl["dt_next"] > 0
    with pf.Simulation(prob, precision=prec) as b:
        b.set_state(u1, t=t1)
        assert b.get_controller()["nhist"] == 0          # set_state starts a fresh controller
        b.set_controller(ctrl)
        assert b.get_controller() == ctrl
        s2b = b.step(integ, t2, tol=TOL, trace_cap=1000)
        ub, tb = b.get_state()
    assert tb == t2
    np.testing.assert_array_equal(s2b["trace"]["dt"], s2["trace"]["dt"])
    np.testing.assert_array_equal(s2b["trace"]["acc"], s2["trace"]["acc"])
    assert np.array_equal(ub, ua)


def test_controller_validation(pf):
    prob, u = I.multiphase_blobs(9, 7, 1, 3, seed=1)
    with pf.Simulation(prob, precision=64) as sim:
        good = {"b": 0.9, "E1": 0.5, "E2": 0.0, "dt1": 0.1, "dt2": 0.0, "dt_next": 0.2, "nhist": 1}
        with pytest.raises(pf.PfError):                  # no state yet
            sim.set_controller(good)
        sim.set_state(u)
        sim.set_controller(good)
        for k, bad in (("b", 0.05), ("b", 1.5), ("nhist", 3), ("E1", -1.0), ("dt_next", float("inf"))):
            with pytest.raises(pf.PfError):
                sim.set_controller(dict(good, **{k: bad}))
