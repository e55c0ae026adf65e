"""Solute conservation of the FP32 path over many stages.

With zero-gradient (or periodic) faces the concentration equation (Eq. ceq)
is in flux form, so sum(c) dV is constant, and every stage of every
integrator is an affine combination of states plus dt times RHS values
(Eq. sts, Alg. ssp2, SSP(10)4), so the total stays constant through a step.
In FP32 the kernels must keep that property up to rounding of the values
themselves: evaluating a0 p0 + a1 v + a2 p2 with FP32-rounded coefficients
scales the total by a factor 1 + O(1e-7) per stage, which compounds to a
loss of per cent over a few hundred thousand stages.  With c stored as
c - c_ref (pf_params.c_ref) the rounding scales with |c - c_ref|, so the
bound shrinks with the share of the domain away from c_ref.
"""
import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

CASES = [
    ("rkl2", 60.0, dict(tol=(1e-4, 1e-4, 1e-4, 1e-4))),
    ("rkl1", 60.0, dict(tol=(1e-4, 1e-4, 1e-4, 1e-4))),
    ("ssp104", 6.0, dict(tol=(1e-4, 1e-4, 1e-4, 1e-4))),
    ("ssp2", 6.0, dict(dt_mult=2.0)),
]


@pytest.mark.parametrize("cref", [0.0, 0.98], ids=["c", "c-0.98"])
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("name,t_end,kw", CASES, ids=[c[0] for c in CASES])
def test_solute_total_is_kept(pf, name, t_end, kw, prec, cref):
    # Bound from the arithmetic: every pass that writes c rounds each cell's
    # stored value (c - c_ref in FP32, c in FP64) once, by at most 2^-p of its
    # magnitude (p = 24 or 53, round to nearest); RKL and SSP(s)2 passes
    # number at most one per RHS evaluation, SSP(10)4 adds two register
    # roundings per ten.  Even if every rounding had the same sign the
    # relative change of sum(c) stays below
    # 1.25 * evaluations * 2^-p * sum|stored| / sum(c).
    prob, u = I.double_triple_junction(nx=96, ny=48, r=16.0, gamma_ab=2.0)
    prob = prob.with_(c_ref=cref)
    integ = I.INTEGRATORS[name]
    N = prob.n_phases
    with pf.Simulation(prob, precision=prec) as sim:
        sim.set_state(u)
        m0 = sim.reduce()[0]
        st = sim.step(integ, t_end, **kw)
        m1 = sim.reduce()[0]
        u1, _ = sim.get_state()
    evals = st["rhs_evals"]
    rel = abs(m1 - m0) / abs(m0)
    shift = cref if prec == 32 else 0.0
    stored = max(np.abs(u[N] - shift).sum(), np.abs(u1[N] - shift).sum()) / u[N].sum()
    bound = 1.25 * evals * 2.0 ** -(24 if prec == 32 else 53) * stored
    print("%s FP%d c_ref %g: %d RHS evaluations, relative change of sum(c) %.3g (bound %.3g)"
          % (name, prec, cref, evals, rel, bound))
    assert evals > 2000
    assert rel <= bound, (rel, bound)
