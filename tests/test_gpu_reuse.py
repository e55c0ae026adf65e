"""Reuse of F(u^{n+1}) as the next step's F(u^n) (PF_STEP_REUSE_RHS).

The stored RHS is the one the next step would evaluate itself, so the
trajectory is the same as without reuse up to rounding; the oracle replays
the attempted (dt, s, accept) sequence.  The RHS count drops by one for every
attempt that follows an accepted one.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import REL64, assert_err_trace, pf, relerr  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _expected_evals(tr):
    acc = tr["acc"]
    reused = int(acc[:-1].sum())            # attempt k > 1 reuses when attempt k - 1 was accepted
    return int((tr["s"] + 1).sum()) - reused


@pytest.mark.parametrize("tol,span", [((1e-4, 1e-3, 1e-4, 1e-4), 60.0), ((1e-6, 1e-6, 1e-6, 1e-6), 4.0)],
                         ids=["tol4", "tol6"])
@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2], ids=["rkl1", "rkl2"])
def test_reuse_replay_fp64(pf, integ, tol, span):
    # tol6 rejects its first attempts: the attempt after a rejection evaluates F again
    prob, u = I.multiphase_blobs(21, 17, 1, 4, seed=11, has_conc=1, n_alpha=1)
    o = ref.Oracle(prob)
    t_end = span * o.dt_e()
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        st = sim.step(integ, t_end, tol=tol, trace_cap=10000, flags=pf.Simulation.STEP_REUSE_RHS)
        ug, tg = sim.get_state()
    tr = st["trace"]
    assert tg == t_end and st["steps_accepted"] >= 3
    assert len(tr["dt"]) == st["steps_accepted"] + st["steps_rejected"] < 10000
    assert st["rhs_evals"] == _expected_evals(tr)
    status, ur, t, trace = o.run(integ, u, 0.0, t_end, tol=tol, replay=(tr["dt"], tr["s"], tr["acc"]),
                                 trace_cap=10000)
    assert status == 0 and t == t_end
    assert_err_trace(trace["err"], tr["err"])
    assert relerr(ug, ur, prob.n_phases, prob.has_conc) <= REL64


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2], ids=["rkl1", "rkl2"])
def test_reuse_same_trajectory(pf, integ, prec):
    prob, u = I.multiphase_blobs(17, 13, 9, 5, seed=3, has_conc=1, n_alpha=2)
    out = []
    for flags in (0, pf.Simulation.STEP_REUSE_RHS):
        with pf.Simulation(prob, precision=prec) as sim:
            sim.set_state(u)
            t_end = 50.0 * sim.dt_e()
            st = sim.step(integ, t_end, tol=(1e-4, 1e-3, 1e-4, 1e-4), trace_cap=4096, flags=flags)
            out.append((st, sim.get_state()[0]))
    (s0, u0), (s1, u1) = out
    for k in ("steps_accepted", "steps_rejected"):
        assert s0[k] == s1[k], k
    np.testing.assert_array_equal(s0["trace"]["s"], s1["trace"]["s"])
    assert s1["rhs_evals"] == _expected_evals(s1["trace"]) < s0["rhs_evals"]
    tol = 1e-12 if prec == 64 else 1e-5
    assert relerr(u1, u0, prob.n_phases, prob.has_conc) <= tol


def test_reuse_across_calls_and_reset(pf):
    # the stored RHS carries over between pf_step calls and is dropped by set_state
    prob, u = I.multiphase_blobs(21, 17, 1, 4, seed=11, has_conc=1, n_alpha=1)
    f = pf.Simulation.STEP_REUSE_RHS
    tol = (1e-4, 1e-3, 1e-4, 1e-4)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        for _ in range(20):                                      # until one attempt is accepted
            a = sim.step(ref.RKL2, 1e30, tol=tol, max_attempts=1, trace_cap=2, flags=f)
            if a["trace"]["acc"][0] == 1:
                break
        assert a["trace"]["acc"][0] == 1
        b = sim.step(ref.RKL2, 1e30, tol=tol, max_attempts=1, trace_cap=2, flags=f)
        assert b["rhs_evals"] == b["trace"]["s"][0]            # stage 1 reused the stored F
        sim.set_state(u)
        c = sim.step(ref.RKL2, 1e30, tol=tol, max_attempts=1, trace_cap=2, flags=f)
        assert c["rhs_evals"] == c["trace"]["s"][0] + 1         # nothing stored after set_state


def test_reuse_ignored_in_masked_storage(pf):
    prob, u = I.multiphase_blobs(17, 13, 9, 5, seed=3, has_conc=1, n_alpha=2)
    out = []
    for flags in (0, pf.Simulation.STEP_REUSE_RHS):
        with pf.Simulation(prob, precision=32, options=pf.Simulation.OPT_MASKED) as sim:
            sim.set_state(u)
            st = sim.step(ref.RKL2, 30 * sim.dt_e(), tol=(1e-4, 1e-3, 1e-4, 1e-4), flags=flags)
            out.append((st["rhs_evals"], sim.get_state()[0]))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
