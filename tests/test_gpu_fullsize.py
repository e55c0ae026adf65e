"""Parity at the benchmark sizes, in the configuration bench.py times, on
sampled cells the oracle can compute one by one.

After one step with s stages a cell's new value depends only on the cells
within s face-neighbour hops.  So the oracle, run on the (2s+1)^d block
around a sampled cell (cut out of the full input, with any boundary
condition of its own), reproduces that cell's new value exactly: errors
from the cut edges travel one cell per stage and do not reach the centre.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16522_gb300 import build
    build.build()
    from paper_2601_16522_gb300 import pf
    return torch, pf


def block(u, shape, centre, r):
    """(2r+1)^d block of u (fields, nz, ny, nx) around centre, periodic wrap."""
    nz, ny, nx = shape
    z, y, x = centre
    uu = u.reshape((u.shape[0],) + shape)
    zi = np.arange(z - r, z + r + 1) % nz if nz > 1 else np.array([0])
    yi = np.arange(y - r, y + r + 1) % ny
    xi = np.arange(x - r, x + r + 1) % nx
    b = uu[:, zi][:, :, yi][:, :, :, xi]
    return np.ascontiguousarray(b.reshape(u.shape[0], -1)), (len(xi), len(yi), len(zi))


def test_grains256_rkl2_step_sampled(env):
    # the bench workload: 256^3, 32 phases, FP32, one RKL2 step of 10 dt_e (s = 7)
    torch, pf = env
    prob, ud = I.grains_device(n=256, n_grains=32, min_dist=40.0, seed=2, dim=3, device="cuda")
    stream = torch.cuda.Stream()
    sim = pf.Simulation(prob, precision=32, stream=stream)
    sim.set_state(ud)
    dte = sim.dt_e()
    dt = 10.0 * dte
    s = ref.sts_stages(ref.RKL2, dt, dte)
    assert s == 7
    sim.step(pf.RKL2, dt, dt_mult=10.0)
    out = torch.empty_like(ud)
    sim.get_state(out=out)
    torch.cuda.synchronize()
    u0 = ud.float().double().cpu().numpy()           # the FP32 values the kernels started from
    u1 = out.cpu().numpy()
    sim.close()
    rng = np.random.default_rng(7)
    # samples: half at interface cells (N_z >= 2 after the step), half anywhere
    phi_max = u1.max(axis=0)
    iface = np.flatnonzero(phi_max < 0.99)
    idx = np.concatenate([rng.choice(iface, 12, replace=False), rng.integers(0, prob.V, 4)])
    worst = 0.0
    for i in idx:
        z, y, x = i // (256 * 256), (i // 256) % 256, i % 256
        ub, (bx, by, bz) = block(u0, (256, 256, 256), (z, y, x), s)
        sub = prob.with_(nx=bx, ny=by, nz=bz)
        o = ref.Oracle(sub)
        assert o.dt_e() == pytest.approx(dte, rel=1e-15)
        un, _, _, _ = o.step(ref.RKL2, dt, s, ub)
        c = ((s * by) + s) * bx + s
        worst = max(worst, np.abs(un[:, c] - u1[:, i]).max())
    # FP32 storage and arithmetic over 7 stages on O(1) fields
    assert worst < 2e-5, worst


def test_stefan_full_fp64_fe_steps_sampled(env):
    # 1024 x 256 Stefan strip, FP64, 6 forward Euler steps at 0.9 dt_e;
    # samples away from the Dirichlet x faces
    torch, pf = env
    prob, u = I.stefan(1024, 256, 200.0)
    with pf.Simulation(prob, precision=64) as sim:
        sim.set_state(u)
        dte = sim.dt_e()
        sim.step(pf.FEULER, 6 * 0.9 * dte, dt_mult=0.9, flags=1)
        u1, _ = sim.get_state()
    rng = np.random.default_rng(8)
    r = 6
    xs = np.concatenate([rng.integers(190, 215, 8), rng.integers(r + 1, 1024 - r - 1, 4)])
    ys = rng.integers(0, 256, len(xs))
    worst = 0.0
    for x, y in zip(xs, ys):
        ub, (bx, by, _) = block(u, (1, 256, 1024), (0, int(y), int(x)), r)
        sub = prob.with_(nx=bx, ny=by, nz=1, bc_phi=(0,) * 6, bc_c=(0,) * 6)   # interior block: any BC
        o = ref.Oracle(sub)
        st, un, t, _ = o.run(ref.FEULER, ub, 0.0, 6 * 0.9 * dte, dt_mult=0.9 * dte / o.dt_e())
        assert st == 0
        c = r * bx + r
        i = y * 1024 + x
        scale = np.abs(u1).max(axis=1)
        worst = max(worst, (np.abs(un[:, c] - u1[:, i]) / scale).max())
    assert worst <= 1e-12, worst
