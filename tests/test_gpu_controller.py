"""Controller and first-stage-fix parity against the oracle.

Controller (Sec. 3.2 stage rule, Sec. 3.3 PID control with bias and reject
fallback, Sec. 5 output times): the GPU run's error norms are fed to the
oracle's own adaptive decision loop (``or_drive``, the loop of ``or_run``
without the model), which must then take the GPU's attempts: the same step
sizes (1e-13 relative: the device-driven loop rounds pow/atan with the GPU
math library), the same RKL stage counts, the same accept flags, across
several output times with the controller state carried between pf_step
calls.  Unlike the replayed trajectories, which force the oracle onto the
GPU's decisions, a wrong exponent, bias update, reject fallback or clip on
the GPU side fails here.

First-stage fix (Sec. 3.2): on a step large enough that the projection acts
on the first RKL2 stage (asserted on the oracle first), the GPU step equals
the oracle's (FP64 at 1e-12; FP32, which multiplies by the reciprocal of
mu~_1 dt, within the FP32 bound)."""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import REL64, pf, relerr  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

TOL = (1e-4, 1e-3, 1e-4, 1e-4)
OUTS = (23.7, 61.0, 97.5)            # output times in units of dt_e


def _stream():
    import torch
    return torch.cuda.Stream()


def _gpu_traces(pf, prob, u, integ, prec, flags, tol=TOL, max_stages=0, dt0=0.0):
    traces = []
    with pf.Simulation(prob, precision=prec, stream=_stream()) as sim:
        sim.set_state(u)
        dte = sim.dt_e()
        for t in OUTS:
            st = sim.step(integ, t * dte, tol=tol, trace_cap=20000, flags=flags,
                          max_stages=max_stages, dt0=dt0)
            assert st["t"] == t * dte
            traces.append(st["trace"])
        dt_next = st["dt_next"]
    return dte, traces, dt_next


def _check_against_drive(integ, dte, traces, dt_next, max_stages=1001, dt0=0.0, own=True):
    """own: the oracle's loop runs on its own step sizes over all output
    times (the host loop uses the same libm, so the sizes agree to the last
    bits); else (device-driven loop, whose pow/atan round as the GPU's math
    library does) each attempt is checked one ahead, continuing from the
    sizes the GPU took: a last-bit difference must not accumulate, because a
    step clipped onto an output time, t_end - t, turns an absolute rounding
    difference of t into a relative one of the (possibly small) step, which
    the controller then carries on."""
    d = ref.Drive(integ, dte, dt0=dt0, max_stages=max_stages)
    n_rej = 0
    for t, tr in zip(OUTS, traces):
        assert len(tr["dt"]) > 0
        np.testing.assert_array_equal(tr["acc"], (tr["err"] < 1.0).astype(np.int32))
        dr = d.run(t * dte, tr["err"], given=None if own else tr["dt"])
        assert len(dr["dt"]) == len(tr["dt"])
        np.testing.assert_array_equal(tr["s"], dr["s"])
        np.testing.assert_array_equal(tr["acc"], dr["acc"])
        # a step clipped onto the output time is t_end - t, where t carries the
        # rounding of the sum of the earlier steps: absolute 1e-13 of t_end
        np.testing.assert_allclose(tr["dt"], dr["dt"], rtol=1e-13, atol=1e-13 * t * dte)
        assert d.t == t * dte
        n_rej += int((tr["acc"] == 0).sum())
    assert d.dt_next == pytest.approx(dt_next, rel=1e-13)
    return n_rej


HOST = 0


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("integ,flags", [
    (ref.RKL1, HOST), (ref.RKL2, HOST), (ref.SSP104, HOST),
    (ref.RKL1, 4), (ref.RKL2, 4),          # PF_STEP_DEVICE_LOOP
    (ref.RKL2, 2),                         # PF_STEP_REUSE_RHS
], ids=["rkl1", "rkl2", "ssp104", "rkl1-devloop", "rkl2-devloop", "rkl2-reuse"])
def test_controller_decisions_match_the_oracle(pf, integ, flags, prec):
    prob, u = I.multiphase_blobs(21, 17, 1, 4, seed=11, has_conc=1, n_alpha=1)
    dte_ref = ref.Oracle(prob).dt_e()
    dte, traces, dt_next = _gpu_traces(pf, prob, u, integ, prec, flags)
    assert dte == pytest.approx(dte_ref, rel=1e-15)
    own = flags != 4                                                  # device loop: one ahead
    assert _check_against_drive(integ, dte, traces, dt_next, own=own) > 0      # rejections included
    if own:
        _check_against_drive(integ, dte, traces, dt_next, own=False)


@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2])
def test_controller_stage_cap_and_rejections_match_the_oracle(pf, integ):
    # loose tolerances and a large first step: the controller asks for steps
    # beyond what 5 stages allow (cut to the cap, not landing on the output
    # time) and rejects attempts (bias squared, reject fallback)
    prob, u = I.multiphase_blobs(19, 15, 1, 3, seed=5, has_conc=1, n_alpha=1)
    tol = (1e-2, 1e-1, 1e-2, 1e-2)
    dte = ref.Oracle(prob).dt_e()
    dte, traces, dt_next = _gpu_traces(pf, prob, u, integ, 64, HOST, tol=tol, max_stages=5, dt0=40.0 * dte)
    assert any((tr["s"] == 5).any() for tr in traces)
    _check_against_drive(integ, dte, traces, dt_next, max_stages=5, dt0=40.0 * dte)
    # the default tolerances from a large first step: the first attempts are
    # rejected until the bias and the reject fallback bring the step down
    dte, traces, dt_next = _gpu_traces(pf, prob, u, integ, 64, HOST, dt0=30.0 * dte)
    assert _check_against_drive(integ, dte, traces, dt_next, dt0=30.0 * dte) > 0


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", ["circle", "blobs"])
def test_rkl2_first_stage_fix_matches_the_oracle(pf, case, prec):
    if case == "circle":
        prob, u = I.circle(24, 6.0, W=1.2)
        mult = 200.0
    else:
        prob, u = I.multiphase_blobs(17, 13, 1, 4, seed=3, has_conc=1, n_alpha=1)
        mult = 120.0
    if prec == 32:
        u = u.astype(np.float32).astype(np.float64)
    o = ref.Oracle(prob)
    dte = o.dt_e()
    dt = mult * dte
    s = ref.sts_stages(ref.RKL2, dt, dte)
    # the projection acts on the first stage u + mu~_1 dt F(u) in some cells
    r0, _ = o.rhs(u)
    mt1 = (4.0 / (s * s + s - 2)) / 3.0
    _, acted, _ = o.project(u + (mt1 * dt) * r0)
    assert acted.sum() > 0
    un_ref, rn_ref, _, _ = o.step(ref.RKL2, dt, s, u)
    assert np.abs(rn_ref - r0).max() > 1e-6          # the effective F(u^n) differs from F(u^n)
    with pf.Simulation(prob, precision=prec) as sim:
        sim.set_state(u)
        st = sim.step(ref.RKL2, dt, dt_mult=mult)
        un, t = sim.get_state()
    assert st["rhs_evals"] == s and t == dt
    N, K = prob.n_phases, prob.has_conc
    if prec == 64:
        assert relerr(un, un_ref, N, K) <= REL64
    else:
        # FP32 storage and stage arithmetic over s stages (s = 29-31 here):
        # a few hundred roundings of 2^-24 of the field scale
        assert relerr(un, un_ref, N, K) <= 2e-5
