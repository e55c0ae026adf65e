"""Slot storage (PF_OPT_SLOTS, Sec. 3.1: at most N_p = 12 phase values and
ids per cell) against the masked one-cell passes, whose arithmetic it
shares (bit for bit while no cell needs more than 12 slots), and against
the oracle's slot rule (or_evict_cell after S) where cells need more."""
import numpy as np
import pytest

from oracle import ref
from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import CASES, pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

SLOTS = 16       # PF_OPT_SLOTS
MASKED = 2       # PF_OPT_MASKED
TOL = (1e-4, 1e-3, 1e-4, 1e-3)
# every case of the parity set whose cells keep at most 12 nonzero values
UNCROWDED = [c for c in CASES if c[0] != "blobs3d_N70"]
# circle32 and stefan have one gamma and one M for every pair (the slot passes
# take the coefficients from the constants); the blobs cases have two chemical
# types with different pair values (the passes gather from the tables)
assert {c[0] for c in UNCROWDED} >= {"circle32", "stefan", "blobs2d_K1", "blobs3d_N33"}


def _run(pf, prob, u, opts, integ, n_dte, **kw):
    with pf.Simulation(prob, precision=32, options=opts) as sim:
        sim.set_state(u)
        st = sim.step(integ, n_dte * sim.dt_e(), **kw)
        out, t = sim.get_state()
    return out, st


@pytest.mark.parametrize("integ,kw", [(ref.FEULER, dict(dt_mult=0.9)), (ref.SSP2, dict(dt_mult=2.0)),
                                      (ref.RKL1, dict(dt_mult=6.0)), (ref.RKL2, dict(dt_mult=12.0))],
                         ids=["fe", "ssp2", "rkl1", "rkl2"])
@pytest.mark.parametrize("name,prob,u", UNCROWDED, ids=[c[0] for c in UNCROWDED])
def test_slots_fixed_steps_equal_masked(pf, name, prob, u, integ, kw):
    n = 10 if integ != ref.FEULER else 6
    masked, st_m = _run(pf, prob, u, MASKED, integ, n, **kw)
    slots, st_s = _run(pf, prob, u, SLOTS, integ, n, **kw)
    assert np.count_nonzero(masked[:prob.n_phases], axis=0).max() <= 12
    assert st_m["rhs_evals"] == st_s["rhs_evals"]
    assert np.array_equal(slots, masked), np.abs(slots - masked).max()


@pytest.mark.parametrize("integ", [ref.RKL1, ref.RKL2], ids=["rkl1", "rkl2"])
@pytest.mark.parametrize("name,prob,u", [UNCROWDED[1], UNCROWDED[3], UNCROWDED[-1]],
                         ids=[UNCROWDED[1][0], UNCROWDED[3][0], UNCROWDED[-1][0]])
def test_slots_adaptive_equal_masked(pf, name, prob, u, integ):
    masked, st_m = _run(pf, prob, u, MASKED, integ, 40, tol=TOL)
    slots, st_s = _run(pf, prob, u, SLOTS, integ, 40, tol=TOL)
    for k in ("rhs_evals", "steps_accepted", "steps_rejected"):
        assert st_m[k] == st_s[k], k
    assert np.array_equal(slots, masked), np.abs(slots - masked).max()


def test_slots_rhs_and_nz(pf):
    name, prob, u = UNCROWDED[3]
    with pf.Simulation(prob, precision=32, options=SLOTS) as sim:
        sim.set_state(u)
        u32, _ = sim.get_state()
        r, nz = sim.rhs()
        _, _, nz2 = sim.get_state(with_nz=True)
    o = ref.Oracle(prob)
    r_ref, nz_ref = o.rhs(u32)
    np.testing.assert_array_equal(nz, nz_ref)
    np.testing.assert_array_equal(nz2, nz_ref)
    N = prob.n_phases
    assert np.abs(r[:N] - r_ref[:N]).max() <= 1e-4 * np.abs(r_ref[:N]).max()


def test_slot_form_round_trip_and_refusals(pf):
    prob, vals, ids, _ = I.grains_slots_device(n=24, n_grains=40, seed=4, device="cpu")
    vals, ids = vals.numpy(), ids.numpy()
    with pf.Simulation(prob, precision=32) as sim:
        sim.set_state_slots(vals, ids, t=2.5)
        v2, i2, c2, t = sim.get_state_slots()
        dense, _ = sim.get_state()
        assert t == 2.5 and c2 is None
        np.testing.assert_array_equal(i2, ids)
        np.testing.assert_array_equal(v2, vals.astype(np.float32).astype(np.float64))
        for k in range(12):
            m = i2[k] >= 0
            np.testing.assert_array_equal(dense[i2[k][m], np.nonzero(m)[0]], v2[k][m])
        assert np.count_nonzero(dense, axis=0).max() == np.count_nonzero(i2 >= 0, axis=0).max()
        # the same state given densely
        sim.set_state(dense)
        v3, i3, _, _ = sim.get_state_slots()
        np.testing.assert_array_equal(i3, i2)
        np.testing.assert_array_equal(v3, v2)
        # an id out of range, a repeated id, thirteen values in one cell
        bad = ids.copy()
        bad[0, 5] = prob.n_phases
        with pytest.raises(RuntimeError):
            sim.set_state_slots(vals, bad)
        bad = ids.copy()
        bad[1, 7] = bad[0, 7]
        vv = vals.copy()
        vv[1, 7] = 0.5
        with pytest.raises(RuntimeError):
            sim.set_state_slots(vv, bad)
        many = np.zeros((13, prob.V))
        mid = np.full((13, prob.V), -1, np.int32)
        many[:, 3] = 1.0 / 13
        mid[:, 3] = np.arange(13)
        many[0, :] = 1.0
        mid[0, :] = 0
        many[0, 3] = 1.0 / 13
        with pytest.raises(RuntimeError):
            sim.set_state_slots(many, mid)
        # integrators and calls without a slot form
        sim.set_state_slots(vals, ids)
        with pytest.raises(RuntimeError):
            sim.step(ref.SSP104, 10 * sim.dt_e(), tol=TOL)
        with pytest.raises(RuntimeError):
            sim.step(ref.RKL2, 10 * sim.dt_e(), tol=TOL, flags=pf.Simulation.STEP_REUSE_RHS)
        with pytest.raises(RuntimeError):
            sim.energy()
    with pytest.raises(RuntimeError):
        pf.Simulation(prob, precision=64)
    with pytest.raises(RuntimeError):
        pf.Simulation(prob, precision=32, options=MASKED)


def _crowded():
    # 20^3 with 100 small grains: six phases per cell at most, but one step
    # brings up to 14 (forward Euler) or 22 (RKL2 at 20 dt_e) nonzero values
    # into single cells
    return I.multiphase_blobs(20, 20, 20, 100, seed=9, has_conc=0, min_dist=3.0)


@pytest.mark.parametrize("integ,mult", [(ref.FEULER, 0.9), (ref.RKL2, 20.0)], ids=["fe", "rkl2"])
def test_slot_rule_against_the_oracle(pf, integ, mult):
    prob, u = _crowded()
    N = prob.n_phases
    with pf.Simulation(prob.with_(n_slots=12), precision=32) as sim:
        sim.set_state(u)
        u32, _ = sim.get_state()
        dt = mult * sim.dt_e()
        st = sim.step(integ, dt, dt_mult=mult, trace_cap=2)
        out, _ = sim.get_state()
    s = int(st["trace"]["s"][0])
    o = ref.Oracle(prob.with_(n_slots=12))
    un, _, _, _ = o.step(integ, dt, s, u32)
    free, _, _, _ = ref.Oracle(prob).step(integ, dt, s, u32)
    assert np.count_nonzero(free[:N], axis=0).max() > 12          # the rule acts
    assert np.count_nonzero(out[:N], axis=0).max() <= 12
    # which phases a cell keeps: the same as the oracle's, up to cells where
    # FP32 rounding reorders two nearly equal values at the cut
    same = ((out[:N] != 0) == (un[:N] != 0)).all(axis=0)
    assert (~same).sum() <= max(1, 2e-3 * prob.V), (~same).sum()
    d = np.abs(out[:N] - un[:N])[:, same]
    assert d.max() <= 2e-5 * s, d.max()
    np.testing.assert_allclose(out[:N].sum(axis=0), 1.0, atol=1e-5)


def test_many_grains_in_slots(pf):
    # 96^3 cells with 600 grains: 12 slots per cell instead of 600 dense
    # planes; adaptive RKL2 keeps every cell on the simplex within its slots
    torch = pytest.importorskip("torch")
    prob, vals, ids, _ = I.grains_slots_device(n=96, n_grains=600, seed=6, device="cuda")
    fp = pf.footprint(prob, 32, options=SLOTS)
    assert fp < 0.05 * 5 * prob.V * 600 * 4
    with pf.Simulation(prob, precision=32, stream=torch.cuda.Stream()) as sim:
        sim.set_state_slots(vals, ids)
        _, _, alive0 = sim.reduce()
        t_end = 50 * sim.dt_e()
        st = sim.step(ref.RKL2, t_end, tol=(1e-4, 1e-2, 1e-4, 1e-4))
        v, i, _, t = sim.get_state_slots(device="cuda")
        _, vol, alive = sim.reduce()
    assert st["steps_accepted"] >= 1 and t == t_end
    assert alive0 == 600 and alive >= 590
    s = v.sum(dim=0)
    assert float((s - 1.0).abs().max()) <= 1e-5
    assert int((i >= 0).sum(dim=0).max()) <= 12
    assert abs(sum(vol) - prob.V * prob.dx ** 3) <= 1e-5 * prob.V * prob.dx ** 3
