"""GPU parity of the energy functional F = int a + w + f dV (Eq. energy).

The CUDA path evaluates F in FP64 whatever the storage precision; it differs
from the oracle only in the order in which the cell energies are summed, so
the totals agree to a few units of FP64 rounding of the sum (bound 1e-12
relative).  FP32 states are compared with the oracle evaluated on the same
FP32-rounded values.
"""
import math

import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import CASES, pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name,prob,u", CASES, ids=[c[0] for c in CASES])
def test_energy_matches_oracle(pf, name, prob, u, prec):
    with pf.Simulation(prob, precision=prec) as sim:
        sim.set_state(u)
        F = sim.energy()
        back, _ = sim.get_state()
    F_ref = ref.Oracle(prob).energy(back)
    assert F_ref > 0.0
    assert abs(F - F_ref) <= REL * abs(F_ref), (F, F_ref)


def test_energy_of_grains_64cubed_32_phases(pf):
    prob, u = I.grains_device(n=64, n_grains=32, min_dist=12.0, seed=2, dim=3, dx=1.0, W_cells=2.5, M=1.0,
                              device="cuda")
    u = u.cpu().numpy()
    with pf.Simulation(prob, precision=32) as sim:
        sim.set_state(u)
        sim.step(pf.RKL2, 5 * sim.dt_e(), tol=(1e-4, 1e-2, 1e-4, 1e-3))
        F = sim.energy()
        back, _ = sim.get_state()
    F_ref = ref.Oracle(prob).energy(back)
    assert abs(F - F_ref) <= REL * abs(F_ref), (F, F_ref)


def test_energy_decreases_along_curvature_flow(pf):
    prob, u = I.circle(128, 40.0, W=5.0 / math.pi)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        dte = sim.dt_e()
        Fs = [sim.energy()]
        for k in range(1, 6):
            sim.step(pf.FEULER, 20 * k * dte, dt_mult=0.9)
            Fs.append(sim.energy())
    assert all(b < a for a, b in zip(Fs, Fs[1:])), Fs
    # the interface energy of a circle of radius 40 is about 2 pi R gamma
    assert Fs[0] == pytest.approx(2 * math.pi * 40.0, rel=0.05)


def test_energy_status(pf):
    prob, u = I.circle(32, 9.0, W=2.5)
    with pf.Simulation(prob, precision=64) as sim:
        with pytest.raises(RuntimeError):
            sim.energy()                      # no state yet
    # more than 32 phases present around one cell is reported, not truncated
    N = 40
    prob = I.Problem(dim=2, nx=16, ny=8, nz=1, dx=1.0, n_phases=N, phase_type=np.zeros(N, np.int32),
                     gamma=I.uniform_pairs(N, 1.0), mobility=I.uniform_pairs(N, 1.0), W=2.5)
    u = np.full((N, prob.V), 1.0 / N)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        with pytest.raises(RuntimeError, match="pf_energy"):
            sim.energy()
