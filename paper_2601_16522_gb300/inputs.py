"""Seeded synthetic inputs: problem descriptions and initial conditions.

This module holds no arithmetic of the time step itself.  It describes a
problem (grid, phases, raw physical parameters, boundary conditions) and builds
initial fields from distance functions, exactly as the paper's benchmark set-up
does (Sec. 4 "Common conditions", Sec. 5).  It is the one piece of code that
both the CUDA engine's callers and the CPU oracle's tests use; it imports only
numpy/scipy.

State layout everywhere: ``u`` of shape ``(N + K, V)`` float64, phase-major,
cell index ``i = (z*ny + y)*nx + x`` (x fastest); row ``N`` is the
concentration when ``K == 1``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET = 0, 1, 2
FEULER, SSP2, SSP104, RKL1, RKL2 = 0, 1, 2, 3, 4
INTEGRATORS = {"feuler": FEULER, "ssp2": SSP2, "ssp104": SSP104, "rkl1": RKL1, "rkl2": RKL2}


@dataclass
class Problem:
    """Raw parameters of one simulation (Sec. 2 model, Sec. 4 parameters)."""
    dim: int
    nx: int
    ny: int
    nz: int
    dx: float
    n_phases: int
    phase_type: np.ndarray          # (N,) int32, chemical type 0 (alpha) or 1 (beta)
    gamma: np.ndarray               # (N, N) interface energies
    mobility: np.ndarray            # (N, N) interface mobilities M
    W: float                        # interface parameter (width pi*W)
    L_override: Optional[np.ndarray] = None   # (N, N) phase-field mobility, e.g. thin-interface L
    has_conc: int = 0
    k: tuple = (1.0, 1.0)
    c0: tuple = (0.0, 0.0)
    D: tuple = (0.0, 0.0)
    bc_phi: tuple = (0, 0, 0, 0, 0, 0)
    bc_c: tuple = (0, 0, 0, 0, 0, 0)
    c_dirichlet: tuple = (0.0,) * 6
    c_ref: float = 0.0              # FP32 storage keeps c - c_ref (the majority phase's c)
    simplex: int = 0                # projection S: 0 standard (Sec. 3.1), 1 mobility-weighted
    n_slots: int = 0                # > 0: per-cell phase slots (Sec. 3.1 N_p), 0: every phase stored
    name: str = ""

    @property
    def V(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nfields(self) -> int:
        return self.n_phases + self.has_conc

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def uniform_pairs(N: int, value: float) -> np.ndarray:
    m = np.full((N, N), float(value))
    np.fill_diagonal(m, 0.0)
    return m


def typed_pairs(ptype, same_beta: float, mixed: float, same_alpha: float = None) -> np.ndarray:
    """Pairwise matrix depending only on the chemical types of the two phases."""
    t = np.asarray(ptype)
    N = len(t)
    m = np.empty((N, N))
    for a in range(N):
        for b in range(N):
            if t[a] != t[b]:
                m[a, b] = mixed
            elif t[a] == 1:
                m[a, b] = same_beta
            else:
                m[a, b] = same_alpha if same_alpha is not None else same_beta
    np.fill_diagonal(m, 0.0)
    return m


# --------------------------------------------------------------------------
# initial profile (Eq. profile) and distance fields
# --------------------------------------------------------------------------

def profile(d, W):
    """Equilibrium 1D profile of Eq. (profile) evaluated on a distance field d."""
    d = np.asarray(d, dtype=np.float64)
    h = math.pi * W / 2.0
    out = 0.5 * (1.0 + np.sin(np.clip(d, -h, h) / W))
    out = np.where(d <= -h, 0.0, out)
    out = np.where(d >= h, 1.0, out)
    return out


def cell_centres(nx, ny, nz, dx):
    """Cell-centred coordinates x_i = (i + 1/2) dx (Sec. 3)."""
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx,
                          (np.arange(nx) + 0.5) * dx, indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


# --------------------------------------------------------------------------
# benchmark problems
# --------------------------------------------------------------------------

def circle(n=128, R0=40.0, W=5.0 / math.pi, M=1.0, gamma=1.0, dx=1.0, ny=None):
    """Shrinking circular grain (Sec. 5.2.1): inner grain = phase 1 with
    distance d = R0 - |X - C| (Eq. centersphere), outer phase 0 = complement.
    2D periodic, phase field only."""
    ny = n if ny is None else ny
    prob = Problem(dim=2, nx=n, ny=ny, nz=1, dx=dx, n_phases=2,
                   phase_type=np.array([0, 0], np.int32),
                   gamma=uniform_pairs(2, gamma), mobility=uniform_pairs(2, M), W=W,
                   name="circle%dx%d" % (n, ny))
    x, y, _ = cell_centres(n, ny, 1, dx)
    cx, cy = n * dx / 2.0, ny * dx / 2.0
    d = R0 - np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    g = profile(d, W)
    u = np.stack([1.0 - g, g])
    return prob, u


def phase_embedding(n=128, r=32.0, W=3.0, D=100.0, k=500.0, c0=(0.02, 0.98), M=1.0, gamma=1.0, dx=1.0):
    """Phase embedding (Sec. 5.1.1): a circle of phase 1 (type beta) of
    radius r (distance d = r - |X - C|, Eq. centersphere) in phase 0 (type
    alpha), both at their flat equilibrium concentrations, c = sum phi_a
    c0_a (mu = 0); 2D periodic, K = 1, equal k (Tab. params), D = 100 as the
    paper uses for equilibrium runs, W = 3 dx^0.4 at dx = 1."""
    prob = Problem(dim=2, nx=n, ny=n, nz=1, dx=dx, n_phases=2, phase_type=np.array([0, 1], np.int32),
                   gamma=uniform_pairs(2, gamma), mobility=uniform_pairs(2, M), W=W, has_conc=1,
                   k=(k, k), c0=tuple(c0), D=(D, D), name="embedding%d" % n)
    x, y, _ = cell_centres(n, n, 1, dx)
    cx = cy = n * dx / 2.0
    g = profile(r - np.sqrt((x - cx) ** 2 + (y - cy) ** 2), W)
    u = np.stack([1.0 - g, g, (1.0 - g) * c0[0] + g * c0[1]])
    return prob, u


def double_triple_junction(nx=192, ny=96, r=32.0, W=2.5, gamma_bb=1.0, gamma_ab=2.0, D=100.0, k=500.0,
                           c0=(0.02, 0.98), M=1.0, dx=1.0, shift=True):
    """Double triple junction (Sec. 5.1.2): a circle of phase 0 (type alpha)
    of radius r centred on the straight boundary y = C_y between grains 1
    (y < C_y) and 2 (type beta), the boundary along the long side.  phi_0
    follows d = r - |X - C| (Eq. centersphere); the grains' trial fields
    profile(C_y - y) and its complement are rescaled to 1 - phi_0 with their
    ratio kept (Eq. distfix).  c is at local equilibrium (mu = 0) and, with
    shift=True, moved uniformly so that its integral equals the sharp-interface
    amount pi r^2 c0_alpha + (area - pi r^2) c0_beta (Sec. 5.1).  Zero-gradient
    faces for phi and c; K = 1, D = 100 and k = 500 as for the paper's
    equilibrium runs."""
    N = 3
    gam = np.array([[0.0, gamma_ab, gamma_ab], [gamma_ab, 0.0, gamma_bb], [gamma_ab, gamma_bb, 0.0]])
    nb = (BC_NEUMANN,) * 4 + (0, 0)
    prob = Problem(dim=2, nx=nx, ny=ny, nz=1, dx=dx, n_phases=N, phase_type=np.array([0, 1, 1], np.int32),
                   gamma=gam, mobility=uniform_pairs(N, M), W=W, has_conc=1, k=(k, k), c0=tuple(c0),
                   D=(D, D), bc_phi=nb, bc_c=nb, c_ref=c0[1], name="triplejunction%dx%d_g%g" % (nx, ny, gamma_ab))
    x, y, _ = cell_centres(nx, ny, 1, dx)
    cx, cy = nx * dx / 2.0, ny * dx / 2.0
    pa = profile(r - np.sqrt((x - cx) ** 2 + (y - cy) ** 2), W)
    t1 = profile(cy - y, W)
    u = np.stack([pa, (1.0 - pa) * t1, (1.0 - pa) * (1.0 - t1), np.zeros_like(pa)])
    u[3] = u[0] * c0[0] + (u[1] + u[2]) * c0[1]
    if shift:
        area = nx * ny * dx * dx
        inner = math.pi * r * r
        target = inner * c0[0] + (area - inner) * c0[1]
        u[3] += (target - u[3].sum() * dx * dx) / area
    return prob, u


def stefan_L(W, k=1.0, dc=0.96, D=1.0, MF=0.3084251):
    """Thin-interface phase-field mobility for vanishing kinetic coefficient
    (Eq. thin-interface, Sec. 5.2.2): L = pi^2/(16 W^2) D (dc/dmu) / (dc_eq^2 (M+F)),
    with dc/dmu = 1/k for the parabolic energies."""
    return (math.pi ** 2 / (16.0 * W * W)) * D * (1.0 / k) / (dc * dc * MF)


def stefan(nx=1024, ny=256, h=200.0, W=5.0 / math.pi, D_liquid=1.0, D_solid=0.01,
           c_liquid=0.2, c_solid=0.98, k=1.0, c0=(0.02, 0.98), dx=1.0, gamma=1.0):
    """Solutal Stefan problem (Sec. 5.2.2) on a 2D strip: solid beta (type 1,
    phase 1) on the left with distance d = h - x, liquid alpha (type 0, phase 0)
    as complement; c = phi_alpha c_liquid + phi_beta c_solid; phi zero-gradient
    on x faces, c Dirichlet (left c_solid, right c_liquid); y periodic."""
    N = 2
    L = stefan_L(W, k=k, dc=c0[1] - c0[0], D=D_liquid)
    Lm = uniform_pairs(N, L)
    prob = Problem(dim=2, nx=nx, ny=ny, nz=1, dx=dx, n_phases=N,
                   phase_type=np.array([0, 1], np.int32),
                   gamma=uniform_pairs(N, gamma), mobility=uniform_pairs(N, 1.0), W=W,
                   L_override=Lm, has_conc=1, k=(k, k), c0=tuple(c0), D=(D_liquid, D_solid),
                   bc_phi=(BC_NEUMANN, BC_NEUMANN, 0, 0, 0, 0),
                   bc_c=(BC_DIRICHLET, BC_DIRICHLET, 0, 0, 0, 0),
                   c_dirichlet=(c_solid, c_liquid, 0.0, 0.0, 0.0, 0.0),
                   name="stefan%dx%d" % (nx, ny))
    x, _, _ = cell_centres(nx, ny, 1, dx)
    solid = profile(h - x, W)
    liquid = 1.0 - solid
    c = liquid * c_liquid + solid * c_solid
    return prob, np.stack([liquid, solid, c])


def stefan_growth_constant(D=1.0, c_a=0.2, c_ab=0.02, c_ba=0.98, c_b=0.98):
    """Root A of Eq. (stefangrowth) by bisection (X(t) = A sqrt(t))."""
    from math import erf, exp, pi, sqrt

    def g(A):
        e = exp(-A * A / (4 * D))
        t1 = (c_a - c_ab) / (c_ba - c_ab) * e / (1 - erf(A / sqrt(4 * D)))
        t2 = (c_b - c_ba) / (c_ba - c_ab) * e / (1 + erf(A / sqrt(4 * D)))
        return sqrt(4 * D / pi) * (t1 + t2) - A

    lo, hi = 1e-9, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(lo) * g(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def poisson_disc_seeds(n_cells, count, min_dist, dim, rng, max_tries=200000):
    """Seeded random points in a periodic box with a minimum (periodic) distance."""
    pts = np.zeros((count, dim))
    n = 0
    tries = 0
    L = np.array(n_cells, dtype=np.float64)
    while n < count:
        tries += 1
        if tries > max_tries:
            raise ValueError("could not place %d seeds with min distance %g" % (count, min_dist))
        p = rng.random(dim) * L
        dd = np.abs(p - pts[:n])
        dd = np.minimum(dd, L - dd)
        if n == 0 or not (np.sqrt((dd * dd).sum(axis=1)) < min_dist).any():
            pts[n] = p
            n += 1
    return pts


def _diffuse_voronoi(shape, seeds, W, knn=6, chunk=1 << 17):
    """Diffuse periodic Voronoi fields: for every grain g among the knn nearest
    seeds, d_g = min over the other neighbours h of the signed distance to the
    bisector of (s_g, s_h); trial phi_g = profile(d_g), rescaled to sum 1
    (the rescaling of Eq. distfix with all trial ratios kept)."""
    from scipy.spatial import cKDTree
    dims = len(shape)
    nz, ny, nx = (shape if dims == 3 else (1,) + tuple(shape))
    G = len(seeds)
    box = np.array([nx, ny, nz][:dims], dtype=np.float64)
    tree = cKDTree(seeds, boxsize=box)
    V = nx * ny * nz
    k = min(knn, G)
    labels_out = np.zeros((k, V), np.int32)
    phis_out = np.zeros((k, V), np.float64)
    eye = np.eye(k, dtype=bool)
    for s0 in range(0, V, chunk):
        idx = np.arange(s0, min(V, s0 + chunk))
        x = idx % nx + 0.5
        y = (idx // nx) % ny + 0.5
        z = idx // (nx * ny) + 0.5
        P = np.stack([x, y, z][:dims], axis=1)
        _, nn = tree.query(P, k=k)
        nn = nn.reshape(len(idx), k)
        S = seeds[nn]                                     # (n, k, dims)
        Dv = P[:, None, :] - S
        Dv -= box * np.round(Dv / box)                    # minimum image
        d2 = (Dv * Dv).sum(-1)                            # (n, k)
        sep = S[:, None, :, :] - S[:, :, None, :]         # (n, g, h, dims)
        sep -= box * np.round(sep / box)
        ln = np.sqrt((sep * sep).sum(-1))
        bis = (d2[:, None, :] - d2[:, :, None]) / (2.0 * np.maximum(ln, 1e-12))
        bis[:, eye] = np.inf
        dist = bis.min(-1)                                # (n, g)
        tr = profile(dist, W)
        tr /= tr.sum(1, keepdims=True)
        labels_out[:, idx] = nn.T
        phis_out[:, idx] = tr.T
    return labels_out, phis_out


def grains(n=256, n_grains=32, min_dist=40.0, seed=2, dim=3, dx=0.005, W_cells=2.5, M=5e-3,
           gamma=1.0, diffuse=True, dtype=np.float64):
    """Periodic Voronoi grain structure (Sec. 5.3): seeded Poisson-disc seeds,
    nearest-seed labelling, dense N = n_grains storage.  diffuse=False gives
    the sharp one-hot start; diffuse=True gives profile-shaped boundaries."""
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    seeds = poisson_disc_seeds(shape, n_grains, min_dist, dim, rng)
    W = W_cells * dx
    prob = Problem(dim=dim, nx=n, ny=n, nz=n if dim == 3 else 1, dx=dx, n_phases=n_grains,
                   phase_type=np.ones(n_grains, np.int32),
                   gamma=uniform_pairs(n_grains, gamma), mobility=uniform_pairs(n_grains, M), W=W,
                   name="grains%d^%d_N%d" % (n, dim, n_grains))
    V = prob.V
    u = np.zeros((n_grains, V), dtype=dtype)
    if diffuse:
        lab, ph = _diffuse_voronoi(shape, seeds, W_cells)
        cols = np.arange(V)
        for j in range(lab.shape[0]):
            u[lab[j], cols] += ph[j]
    else:
        from scipy.spatial import cKDTree
        tree = cKDTree(seeds, boxsize=np.full(dim, float(n)))
        x, y, z = cell_centres(prob.nx, prob.ny, prob.nz, 1.0)
        P = np.stack([x, y, z][:dim], axis=1)
        _, lab = tree.query(P, k=1)
        u[lab, np.arange(V)] = 1.0
    return prob, u


def multiphase_blobs(nx=24, ny=20, nz=1, n_phases=5, seed=0, W=1.6, dx=1.0, has_conc=0,
                     n_alpha=1, k=(1.0, 1.0), c0=(0.02, 0.98), D=(1.0, 0.5), M=1.0,
                     gamma=1.0, bc_phi=(0,) * 6, bc_c=(0,) * 6, c_dirichlet=(0.0,) * 6,
                     min_dist=None):
    """Small seeded diffuse multi-grain state with triple junctions, used for
    parity tests on odd grid sizes.  Phases 0..n_alpha-1 have type alpha."""
    rng = np.random.default_rng(seed)
    dim = 2 if nz == 1 else 3
    shape = (nx, ny) if dim == 2 else (nx, ny, nz)
    md = min_dist if min_dist is not None else 0.5 * (np.prod(shape) / n_phases) ** (1.0 / dim)
    seeds = poisson_disc_seeds(shape, n_phases, md, dim, rng)
    lab, ph = _diffuse_voronoi(shape[::-1] if dim == 3 else (ny, nx), seeds, W / dx)
    V = nx * ny * nz
    ptype = np.array([0 if a < n_alpha else 1 for a in range(n_phases)], np.int32)
    gam = typed_pairs(ptype, gamma, 1.3 * gamma)
    mob = typed_pairs(ptype, M, 0.7 * M)
    prob = Problem(dim=dim, nx=nx, ny=ny, nz=nz, dx=dx, n_phases=n_phases, phase_type=ptype,
                   gamma=gam, mobility=mob, W=W, has_conc=has_conc, k=tuple(k), c0=tuple(c0),
                   D=tuple(D), bc_phi=tuple(bc_phi), bc_c=tuple(bc_c),
                   c_dirichlet=tuple(c_dirichlet), name="blobs%dx%dx%d_N%d" % (nx, ny, nz, n_phases))
    u = np.zeros((n_phases + has_conc, V))
    cols = np.arange(V)
    for j in range(lab.shape[0]):
        u[lab[j], cols] += ph[j]
    if has_conc:
        # local equilibrium c = sum_a phi_a c0_a plus a seeded smooth perturbation
        x, y, z = cell_centres(nx, ny, nz, 1.0)
        pert = 0.02 * np.sin(2 * np.pi * x / nx + rng.random() * 6) * np.cos(2 * np.pi * y / ny)
        c = sum(u[a] * c0[ptype[a]] for a in range(n_phases)) + pert
        u[n_phases] = c
    return prob, u


def grains_device(n=256, n_grains=32, min_dist=40.0, seed=2, dim=3, dx=0.005, W_cells=2.5, M=5e-3,
                  gamma=1.0, knn=6, device="cuda", chunk=1 << 20, region=None):
    """Same structure as grains(diffuse=True), built with torch on a device
    (brute-force nearest seeds): returns (Problem, u) with u a float64 tensor
    of shape (n_grains, V) on `device`.  Used for large benchmark inputs.
    region=m evaluates only the corner m^dim block (u then has m^dim columns,
    ordered x-fastest within the block) of the full n^dim structure."""
    import torch
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    seeds = poisson_disc_seeds(shape, n_grains, min_dist, dim, rng)
    W = W_cells * dx
    prob = Problem(dim=dim, nx=n, ny=n, nz=n if dim == 3 else 1, dx=dx, n_phases=n_grains,
                   phase_type=np.ones(n_grains, np.int32),
                   gamma=uniform_pairs(n_grains, gamma), mobility=uniform_pairs(n_grains, M), W=W,
                   name="grains%d^%d_N%d" % (n, dim, n_grains))
    m = n if region is None else region
    V = m ** dim
    u = torch.zeros((n_grains, V), dtype=torch.float64, device=device)
    for idx, nn, tr in _voronoi_chunks(seeds, n, m, dim, W_cells, knn, device, chunk):
        for j in range(nn.shape[1]):
            u.index_put_((nn[:, j], idx), tr[:, j], accumulate=True)
    return prob, u


def _voronoi_chunks(seeds, n, m, dim, W_cells, knn, device, chunk):
    """The diffuse periodic Voronoi structure of grains_device, chunk by
    chunk of cells: yields (cell indices, the k nearest seeds per cell, their
    trial values rescaled to sum 1)."""
    import torch
    V = m ** dim
    S = torch.tensor(seeds, dtype=torch.float64, device=device)
    box = torch.full((dim,), float(n), dtype=torch.float64, device=device)
    k = min(knn, len(seeds))
    eye = torch.eye(k, dtype=torch.bool, device=device)
    h = math.pi * W_cells / 2.0
    for s0 in range(0, V, chunk):
        idx = torch.arange(s0, min(V, s0 + chunk), device=device)
        coords = [idx % m + 0.5, (idx // m) % m + 0.5, idx // (m * m) + 0.5][:dim]
        P = torch.stack([c.to(torch.float64) for c in coords], dim=1)
        Dv = P[:, None, :] - S[None]
        Dv -= box * torch.round(Dv / box)
        d2all = (Dv * Dv).sum(-1)
        d2, nn = torch.topk(d2all, k, dim=1, largest=False)
        Sk = S[nn]
        sep = Sk[:, None, :, :] - Sk[:, :, None, :]
        sep -= box * torch.round(sep / box)
        ln = torch.sqrt((sep * sep).sum(-1)).clamp_min(1e-12)
        bis = (d2[:, None, :] - d2[:, :, None]) / (2.0 * ln)
        bis[:, eye] = float("inf")
        dist = bis.min(-1).values
        tr = 0.5 * (1.0 + torch.sin(dist.clamp(-h, h) / W_cells))
        tr = torch.where(dist <= -h, torch.zeros_like(tr), tr)
        tr = torch.where(dist >= h, torch.ones_like(tr), tr)
        tr /= tr.sum(1, keepdim=True)
        yield idx, nn, tr


N_SLOTS = 12    # per-cell phase slots of the slot storage (Sec. 3.1: N_p = 12)


def grains_slots_device(n=256, n_grains=2000, min_dist=None, seed=2, dim=3, dx=0.005, W_cells=2.5, M=5e-3,
                        gamma=1.0, knn=6, device="cuda"):
    """The grain structure of grains_device with many grains, returned in
    per-cell slot form (Sec. 3.1: each cell holds its nonzero phase values
    with their phase ids, at most N_SLOTS): (Problem, vals, ids, None) with
    vals a (N_SLOTS, V) float64 tensor and ids a (N_SLOTS, V) int32 tensor,
    slots in ascending id order, -1 (value 0) where empty.  min_dist defaults
    to 0.6 of the mean grain spacing."""
    import torch
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    if min_dist is None:
        min_dist = 0.6 * (n ** dim / n_grains) ** (1.0 / dim)
    seeds = poisson_disc_seeds(shape, n_grains, min_dist, dim, rng, max_tries=50 * n_grains + 200000)
    W = W_cells * dx
    prob = Problem(dim=dim, nx=n, ny=n, nz=n if dim == 3 else 1, dx=dx, n_phases=n_grains,
                   phase_type=np.ones(n_grains, np.int32),
                   gamma=uniform_pairs(n_grains, gamma), mobility=uniform_pairs(n_grains, M), W=W,
                   n_slots=N_SLOTS, name="grains%d^%d_N%d_slots" % (n, dim, n_grains))
    V = n ** dim
    vals = torch.zeros((N_SLOTS, V), dtype=torch.float64, device=device)
    ids = torch.full((N_SLOTS, V), -1, dtype=torch.int32, device=device)
    chunk = max(1024, (1 << 25) // n_grains)
    for idx, nn, tr in _voronoi_chunks(seeds, n, n, dim, W_cells, knn, device, chunk):
        # ascending ids, zero trial values left out (they sort after the others)
        key = torch.where(tr > 0, nn, torch.full_like(nn, 1 << 30))
        key, order = torch.sort(key, dim=1)
        tv = torch.gather(tr, 1, order)
        k = nn.shape[1]
        vals[:k, idx] = torch.where(key < (1 << 30), tv, torch.zeros_like(tv)).T
        ids[:k, idx] = torch.where(key < (1 << 30), key, torch.full_like(key, -1)).to(torch.int32).T
    return prob, vals, ids, None


def corrected_radius(r, W, tol=1e-10):
    """Radius r_c whose diffuse sphere (Eq. profile of r_c - |x|) holds the
    sharp volume 4/3 pi r^3 (the radius correction of Sec. 5.3, solved here by
    bisection on the continuous volume integral)."""
    h = math.pi * W / 2.0

    def vol(rc):
        rho = np.linspace(0.0, rc + h, 4001)
        return 4.0 * math.pi * np.trapezoid(rho ** 2 * profile(rc - rho, W), rho)

    target = 4.0 / 3.0 * math.pi * r ** 3
    lo, hi = 0.0, r + h
    while hi - lo > tol * max(1.0, r):
        mid = 0.5 * (lo + hi)
        if vol(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def sintering_device(n=320, n_grains=64, porosity=0.05, r_range=(4.0, 8.0), gap=4.0, seed=3, dx=0.005,
                     W_cells=2.5, M_gb=5e-3, M_gp=5e-3, D_pore=10.0, D_grain=5e-8, k=1e5, c0=(0.02, 0.98),
                     gamma=1.0, grain_min_dist=None, device="cuda"):
    """Final-stage sintering state (Sec. 5.3, mobile pores): a periodic
    Voronoi grain structure (grains: type beta, phases 0..n_grains-1) with
    spherical pores (one pore phase of type alpha, last phase) of radii
    U[r_range] cells placed at seeded sites whose centres are at least
    r_i + r_j + 2 gap apart, until the sharp pore volume reaches `porosity`.
    Pores use the corrected radius, grains are rescaled by (1 - phi_pore)
    (Eq. distfix with the ratios kept), and c is at local equilibrium
    c = sum_a phi_a c0_a.  Returns (Problem, u) with u a float64 device tensor."""
    import torch
    rng = np.random.default_rng(seed)
    gmd = grain_min_dist if grain_min_dist is not None else 0.8 * n / n_grains ** (1.0 / 3.0)
    prob_g, ug = grains_device(n=n, n_grains=n_grains, min_dist=gmd, seed=seed, dim=3, dx=dx, W_cells=W_cells,
                               M=M_gb, gamma=gamma, device=device)
    V = n ** 3
    target = porosity * V
    centres, radii = [], []
    vol = 0.0
    tries = 0
    while vol < target:
        tries += 1
        if tries > 2000000:
            raise ValueError("cannot reach porosity %g" % porosity)
        c = rng.random(3) * n
        r = rng.uniform(*r_range)
        if centres:
            d = np.abs(np.array(centres) - c)
            d = np.minimum(d, n - d)
            if np.any(np.sqrt((d * d).sum(1)) < np.array(radii) + r + 2.0 * gap):
                continue
        centres.append(c)
        radii.append(r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    # pore phase: max over pores of profile(r_c - |x - s|), stamped box by box
    h = math.pi * W_cells / 2.0
    phip = torch.zeros(V, dtype=torch.float64, device=device)
    rc_cache = {}
    for c, r in zip(centres, radii):
        rc = corrected_radius(r, W_cells)
        R = int(math.ceil(rc + h)) + 1
        off = torch.arange(-R, R + 1, device=device)
        zz, yy, xx = torch.meshgrid(off, off, off, indexing="ij")
        ci = np.floor(c).astype(int)
        X = (ci[0] + xx) % n
        Y = (ci[1] + yy) % n
        Z = (ci[2] + zz) % n
        dxv = (ci[0] + xx + 0.5 - c[0]).double()
        dyv = (ci[1] + yy + 0.5 - c[1]).double()
        dzv = (ci[2] + zz + 0.5 - c[2]).double()
        d = rc - torch.sqrt(dxv * dxv + dyv * dyv + dzv * dzv)
        val = 0.5 * (1.0 + torch.sin(d.clamp(-h, h) / W_cells))
        val = torch.where(d <= -h, torch.zeros_like(val), val)
        val = torch.where(d >= h, torch.ones_like(val), val)
        idx = ((Z * n + Y) * n + X).reshape(-1)
        phip.scatter_reduce_(0, idx, val.reshape(-1), reduce="amax")
    N = n_grains + 1
    u = torch.empty((N + 1, V), dtype=torch.float64, device=device)
    u[:n_grains] = ug * (1.0 - phip)[None, :]
    u[n_grains] = phip
    u[N] = c0[0] * phip + c0[1] * (1.0 - phip)
    ptype = np.ones(N, np.int32)
    ptype[n_grains] = 0
    prob = Problem(dim=3, nx=n, ny=n, nz=n, dx=dx, n_phases=N, phase_type=ptype,
                   gamma=uniform_pairs(N, gamma), mobility=typed_pairs(ptype, M_gb, M_gp), W=W_cells * dx,
                   has_conc=1, k=(k, k), c0=tuple(c0), D=(D_pore, D_grain), c_ref=c0[1],
                   name="sinter%d^3_N%d_pores%d" % (n, N, len(centres)))
    prob.pores = len(centres)
    prob.porosity = float(phip.sum().item()) / V
    return prob, u


def zener_device(n=320, n_grains=64, fraction=0.15, r=6.0, seed=5, dx=0.005, W_cells=2.5, device="cuda"):
    """Grain growth with immobile particles (Sec. 5.3, Zener pinning): the
    sintering construction with particles of one radius r = 6 cells at volume
    fraction 0.15 whose centres are at least 2 r apart, and the immobile
    parameters M_ab = D_alpha = 5e-8 (M_bb = 5e-3, D_beta = 5e-8, k = 1e5).
    Returns (Problem, u) with u a float64 device tensor."""
    prob, u = sintering_device(n=n, n_grains=n_grains, porosity=fraction, r_range=(r, r), gap=0.0, seed=seed,
                               dx=dx, W_cells=W_cells, M_gb=5e-3, M_gp=5e-8, D_pore=5e-8, D_grain=5e-8,
                               k=1e5, device=device)
    prob.name = "zener%d^3_N%d_particles%d" % (n, prob.n_phases, prob.pores)
    return prob, u


def zener_equilibration(prob):
    """Parameters of the equilibration run that precedes the particle runs
    (Sec. 5.3): M_bb = 5e-8, M_ab = 5e-3, D_alpha = 5e-3 (D_beta kept), run
    for 5 time units so that the particles relax capillarily while the grains
    barely move."""
    pt = prob.phase_type
    out = prob.with_(mobility=typed_pairs(pt, 5e-8, 5e-3), D=(5e-3, prob.D[1]),
                     name=prob.name + "_equilibration")
    for a in ("pores", "porosity"):
        if hasattr(prob, a):
            setattr(out, a, getattr(prob, a))
    return out
