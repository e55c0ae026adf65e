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


def test_poisson_disc_seeds_keep_their_periodic_distance():
    rng = np.random.default_rng(3)
    pts = I.poisson_disc_seeds((40, 30, 20), 25, 7.0, 3, rng)
    assert pts.shape == (25, 3)
    L = np.array([40.0, 30.0, 20.0])
    assert np.all(pts >= 0) and np.all(pts < L)
    d = np.abs(pts[:, None, :] - pts[None, :, :])
    d = np.minimum(d, L - d)
    dist = np.sqrt((d * d).sum(-1)) + np.eye(25) * 1e9
    assert dist.min() >= 7.0
    with pytest.raises(ValueError):                      # cannot be placed: refused, not looped forever
        I.poisson_disc_seeds((10, 10), 50, 6.0, 2, np.random.default_rng(0), max_tries=2000)


def test_corrected_radius_gives_the_sharp_volume():
    # Sec. 5.3: the diffuse sphere of radius r_c holds the sharp volume 4/3 pi r^3
    # (checked here on a fine cell grid, independently of the builder's quadrature)
    W = 2.5
    for r in (4.0, 6.0, 8.0):
        rc = I.corrected_radius(r, W)
        assert rc < r
        h = 0.25
        n = int(np.ceil((rc + math.pi * W / 2 + 1) / h))
        ax = (np.arange(-n, n) + 0.5) * h
        X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
        vol = I.profile(rc - np.sqrt(X * X + Y * Y + Z * Z), W).sum() * h ** 3
        assert vol == pytest.approx(4.0 / 3.0 * math.pi * r ** 3, rel=2e-3)


def test_diffuse_voronoi_grains_are_a_partition():
    prob, u = I.grains(n=24, n_grains=6, min_dist=8.0, seed=4, dim=3, dx=1.0, W_cells=2.5, M=1.0)
    np.testing.assert_allclose(u.sum(0), 1.0, atol=1e-14)
    assert u.min() >= 0.0 and u.max() <= 1.0
    assert (u.max(1) >= 0.5).sum() == 6                    # every grain has a bulk
    # bulk cells (one phase at exactly 1) exist, and no cell holds more than
    # the knn = 6 nearest grains the construction considers
    assert (u == 1.0).any(axis=0).any()
    assert (u > 0).sum(0).max() <= 6


def test_slot_form_grains_are_the_dense_grains():
    # the slot form lists, per cell, the nonzero values of the dense builder's
    # state in ascending phase order (the same seeds and profiles)
    pytest.importorskip("torch")
    prob_d, u = I.grains_device(n=20, n_grains=12, min_dist=5.0, seed=3, dim=3, device="cpu")
    prob_s, vals, ids, _ = I.grains_slots_device(n=20, n_grains=12, min_dist=5.0, seed=3, dim=3, device="cpu")
    u, vals, ids = u.numpy(), vals.numpy(), ids.numpy()
    assert prob_s.n_slots == I.N_SLOTS and prob_s.n_phases == prob_d.n_phases
    dense = np.zeros_like(u)
    for k in range(I.N_SLOTS):
        m = ids[k] >= 0
        dense[ids[k][m], np.nonzero(m)[0]] = vals[k][m]
        assert np.all(vals[k][~m] == 0.0)
    np.testing.assert_array_equal(dense, u)
    used = ids >= 0
    assert np.all(used[:-1] | ~used[1:])                      # used slots come first
    d = np.diff(np.where(used, ids, 1 << 30), axis=0)
    assert np.all((d > 0) | ~used[1:])                        # ascending ids
    assert np.count_nonzero(u, axis=0).max() == used.sum(axis=0).max()
