"""The seeded input builders against what their sections of the paper fix
(construction only; no step of the method)."""
import math

import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I


def test_double_triple_junction_construction():
    # Sec. 5.1.2: the lens follows Eq. centersphere exactly, the two grains
    # keep the ratio of their trial fields (Eq. distfix) and fill 1 - phi_0,
    # c sits at local equilibrium shifted uniformly to the sharp-interface
    # amount pi r^2 c0_alpha + (area - pi r^2) c0_beta (Sec. 5.1).
    r = 32.0
    prob, u = I.double_triple_junction(r=r, gamma_ab=2.0)
    nx, ny = prob.nx, prob.ny
    x, y, _ = I.cell_centres(nx, ny, 1, 1.0)
    lens = I.profile(r - np.hypot(x - nx / 2, y - ny / 2), prob.W)
    np.testing.assert_allclose(u[0], lens, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[:3].sum(0), 1.0, atol=1e-15)
    t1 = I.profile(ny / 2 - y, prob.W)
    both = (u[1] > 0) & (u[2] > 0)
    np.testing.assert_allclose(u[1][both] / u[2][both], t1[both] / (1 - t1[both]), rtol=1e-12)
    sharp = math.pi * r * r * 0.02 + (nx * ny - math.pi * r * r) * 0.98
    assert u[3].sum() == pytest.approx(sharp, rel=1e-14)
    shift = u[3] - (0.02 * u[0] + 0.98 * (u[1] + u[2]))
    assert np.ptp(shift) < 1e-14                           # one uniform shift
    assert prob.gamma[0, 1] == prob.gamma[0, 2] == 2.0 and prob.gamma[1, 2] == 1.0
    assert all(b == I.BC_NEUMANN for b in prob.bc_phi[:4]) and prob.bc_c == prob.bc_phi
    unshifted = I.double_triple_junction(r=r, gamma_ab=2.0, shift=False)[1]
    np.testing.assert_allclose(unshifted[3], 0.02 * u[0] + 0.98 * (u[1] + u[2]), atol=1e-15)


def test_zener_construction_and_equilibration_parameters():
    # Sec. 5.3: particles of one radius at volume fraction 0.15 with the
    # immobile parameters; the equilibration run changes only M_bb, M_ab
    # and D_alpha.
    prob, u = I.zener_device(n=48, n_grains=8, device="cpu")
    u = u.numpy()
    N = prob.n_phases
    assert N == 9 and list(prob.phase_type) == [1] * 8 + [0]
    assert abs(prob.porosity - 0.15) < 0.01
    np.testing.assert_allclose(u[:N].sum(0), 1.0, atol=1e-14)
    assert u[:N].min() >= 0.0
    np.testing.assert_allclose(u[N], 0.02 * u[N - 1] + 0.98 * (1.0 - u[N - 1]), atol=1e-15)
    assert prob.mobility[0, 1] == 5e-3 and prob.mobility[0, N - 1] == 5e-8
    assert prob.D == (5e-8, 5e-8) and prob.k == (1e5, 1e5)
    eq = I.zener_equilibration(prob)
    assert eq.mobility[0, 1] == 5e-8 and eq.mobility[0, N - 1] == 5e-3
    assert eq.D == (5e-3, 5e-8)
    for f in ("gamma", "W", "k", "c0", "dx", "n_phases"):
        assert np.array_equal(np.asarray(getattr(eq, f)), np.asarray(getattr(prob, f)))
