"""FP32 storage of c relative to a reference concentration (pf_params.c_ref).

The engine keeps c - c_ref in FP32 and shifts c0 and the Dirichlet values by
the same amount, so mu = (c - sum phi c0) / (sum phi / k), the face fluxes of
Eq. ceq and every difference of psi in Eq. phieq are those of c; only the
error weights |c| add c_ref back.  The results therefore match the FP64
oracle as closely as with c_ref = 0, the state and totals come back as c,
and values near c_ref keep FP32's relative resolution.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import CASES, pf, relerr  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

K1 = [CASES[1], CASES[2], CASES[3], CASES[5]]      # CASES[2]: a Dirichlet c face


@pytest.mark.parametrize("name,prob,u", K1, ids=[c[0] for c in K1])
def test_rhs_fp32_with_c_ref(pf, name, prob, u):
    # same bound as without the shift (FP32 rounding amplified by the mu
    # cancellation and the flux differences)
    u = u.astype(np.float32).astype(np.float64)
    r_ref, nz_ref = ref.Oracle(prob).rhs(u)
    with pf.Simulation(prob.with_(c_ref=0.98), precision=32) as sim:
        sim.set_state(u)
        r, nz = sim.rhs()
    assert relerr(r, r_ref, prob.n_phases, prob.has_conc) < 1e-3
    np.testing.assert_array_equal(nz, nz_ref)


@pytest.mark.parametrize("integ,mult", [(ref.RKL2, 8.0), (ref.SSP2, 2.0), (ref.FEULER, 0.9)],
                         ids=["rkl2", "ssp2", "fe"])
def test_step_fp32_with_c_ref(pf, integ, mult):
    name, prob, u = CASES[5]
    u = u.astype(np.float32).astype(np.float64)
    o = ref.Oracle(prob)
    dte = o.dt_e()
    s = ref.sts_stages(integ, mult * dte, dte) if integ == ref.RKL2 else 5
    un_ref, _, _, _ = o.step(integ, mult * dte, s, u)
    with pf.Simulation(prob.with_(c_ref=0.98), precision=32) as sim:
        sim.set_state(u)
        sim.step(integ, mult * dte, dt_mult=mult)
        ug, _ = sim.get_state()
    assert relerr(ug, un_ref, prob.n_phases, prob.has_conc) < 1e-4


def test_state_and_totals_come_back_as_c(pf):
    name, prob, u = CASES[3]
    N = prob.n_phases
    cref = 0.98
    with pf.Simulation(prob.with_(c_ref=cref), precision=32) as sim:
        sim.set_state(u)
        ug, _ = sim.get_state()
        mass, vol, _ = sim.reduce()
    stored = (u[N] - cref).astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(ug[N], stored + cref)
    dv = prob.dx ** prob.dim
    assert mass == pytest.approx(ug[N].sum() * dv, rel=1e-12)
    # near c_ref the stored value keeps its own relative resolution
    near = np.abs(u[N] - cref) < 1e-2
    assert near.any()
    assert np.abs(ug[N] - u[N])[near].max() <= 2.0 ** -24 * 1e-2


def test_c_ref_ignored_in_fp64(pf):
    name, prob, u = CASES[1]
    out = []
    for cref in (0.0, 0.98):
        with pf.Simulation(prob.with_(c_ref=cref), precision=64) as sim:
            sim.set_state(u)
            sim.step(ref.RKL2, 10 * sim.dt_e(), dt_mult=10.0)
            out.append(sim.get_state()[0])
    assert np.array_equal(out[0], out[1])


def test_non_finite_c_ref_is_rejected(pf):
    name, prob, u = CASES[1]
    with pytest.raises(pf.PfError):
        pf.Simulation(prob.with_(c_ref=float("nan")), precision=32)
