"""Device-driven adaptive RKL steps (PF_STEP_DEVICE_LOOP: a CUDA graph with
conditional WHILE nodes, every controller decision on the GPU) against the
FP64 oracle and against the host-driven loop.

The oracle replays the attempted (dt, s, accept) sequence the GPU chose, so
parity is checked exactly as for the host loop.  Against the host loop the
only difference is the rounding of pow/atan in the controller (GPU math
library vs the host's), so the attempt sequences agree and the states agree
to rounding.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import REL64, assert_err_trace, pf, relerr  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

TOL = (1e-4, 1e-3, 1e-4, 1e-4)


def _stream():
    import torch
    return torch.cuda.Stream()


def _device_launches(trace, graph_launches, kpp=1):
    # per attempt: plan + stage 1, (s - 1) x (plan + stage), plan + error
    # sweep, norm, controller; plus one begin kernel per graph launch.  kpp:
    # kernels per pass (2 for the FP32 two-cell passes: the pass and the wide
    # pass of its crowded cells)
    return int(np.sum((trace["s"] + 1) * (1 + kpp) + 2)) + graph_launches


@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2], ids=["rkl1", "rkl2"])
def test_devloop_replay_fp64(pf, integ):
    prob, u = I.multiphase_blobs(21, 17, 1, 4, seed=11, has_conc=1, n_alpha=1)
    o = ref.Oracle(prob)
    t_end = 60.0 * o.dt_e()
    with pf.Simulation(prob, precision=64, stream=_stream()) as sim:
        sim.set_state(u)
        st = sim.step(integ, t_end, tol=TOL, trace_cap=10000, flags=pf.Simulation.STEP_DEVICE_LOOP)
        ug, tg = sim.get_state()
    tr = st["trace"]
    assert tg == t_end
    assert st["steps_accepted"] >= 3
    assert st["kernel_launches"] == _device_launches(tr, 1)      # the device-driven loop ran
    status, ur, t, trace = o.run(integ, u, 0.0, t_end, tol=TOL, replay=(tr["dt"], tr["s"], tr["acc"]),
                                 trace_cap=10000)
    assert status == 0 and t == t_end
    assert_err_trace(trace["err"], tr["err"])
    assert relerr(ug, ur, prob.n_phases, prob.has_conc) <= REL64
    assert st["rhs_evals"] == o.stats.rhs_evals


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2], ids=["rkl1", "rkl2"])
def test_devloop_matches_host_loop(pf, integ, prec):
    prob, u = I.multiphase_blobs(17, 13, 9, 5, seed=3, has_conc=1, n_alpha=2)
    out = []
    for flags in (pf.Simulation.STEP_DEVICE_LOOP, 0):
        with pf.Simulation(prob, precision=prec, stream=_stream()) as sim:
            sim.set_state(u)
            t_end = 50.0 * sim.dt_e()
            st = sim.step(integ, t_end, tol=TOL, trace_cap=4096, flags=flags)
            out.append((st, sim.get_state()[0]))
    (sd, ud), (sh, uh) = out
    for k in ("steps_accepted", "steps_rejected", "rhs_evals", "t"):
        assert sd[k] == sh[k], k
    np.testing.assert_array_equal(sd["trace"]["s"], sh["trace"]["s"])
    np.testing.assert_allclose(sd["trace"]["dt"], sh["trace"]["dt"], rtol=1e-12)
    tol = 1e-10 if prec == 64 else 1e-5
    assert relerr(ud, uh, prob.n_phases, prob.has_conc) <= tol


def test_devloop_several_graph_launches(pf):
    # more than 256 attempts: the host relaunches the graph until t_end
    prob, u = I.circle(64, 20.0, W=2.5)
    tol = (1e-6, 1e-6, 1e-6, 1e-6)
    with pf.Simulation(prob, precision=32, stream=_stream()) as sim:
        sim.set_state(u)
        t_end = 3000.0 * sim.dt_e()
        st = sim.step(ref.RKL2, t_end, tol=tol, trace_cap=100000, flags=pf.Simulation.STEP_DEVICE_LOOP)
        ug, tg = sim.get_state()
    n = len(st["trace"]["dt"])
    assert n > 256
    assert tg == t_end
    assert st["kernel_launches"] == _device_launches(st["trace"], (n + 255) // 256, kpp=2)
    with pf.Simulation(prob, precision=32, stream=_stream()) as sim:
        sim.set_state(u)
        sh = sim.step(ref.RKL2, t_end, tol=tol)
        uh, _ = sim.get_state()
    assert abs(st["steps_accepted"] - sh["steps_accepted"]) <= 2
    assert relerr(ug, uh, prob.n_phases, prob.has_conc) <= 1e-4


def test_devloop_max_attempts_resume_and_eligibility(pf):
    prob, u = I.multiphase_blobs(21, 17, 1, 4, seed=11, has_conc=1, n_alpha=1)
    f = pf.Simulation.STEP_DEVICE_LOOP
    with pf.Simulation(prob, precision=64, stream=_stream()) as sim:
        sim.set_state(u)
        t_end = 60.0 * sim.dt_e()
        st1 = sim.step(ref.RKL2, t_end, tol=TOL, max_attempts=1, trace_cap=4, flags=f)
        assert st1["steps_accepted"] + st1["steps_rejected"] == 1
        st2 = sim.step(ref.RKL2, t_end, tol=TOL, trace_cap=10000, flags=f)
        ug, tg = sim.get_state()
        # the controller state carries over to the next call
        assert st2["trace"]["dt"][0] == pytest.approx(st1["dt_next"], rel=1e-15)
        assert tg == t_end
        with pytest.raises(RuntimeError):                          # fixed steps have no device loop
            sim.step(ref.RKL2, 2 * t_end, dt_mult=4.0, flags=f)
    with pf.Simulation(prob, precision=64) as sim:                 # the default stream cannot be captured
        sim.set_state(u)
        with pytest.raises(RuntimeError):
            sim.step(ref.RKL2, 10 * sim.dt_e(), tol=TOL, flags=f)
