"""Batched stepping (pf_batch_*) and the caller-supplied allocator.

Each request admitted into a batch must end exactly where pf_step on the same
handle alone ends: the same state bit for bit, the same time, RHS count and
accepted/rejected attempts.  The mix covers packed requests (FP32 dense, nx
even: 2D/3D, K = 0/1, fixed FE/SSP(5)2/RKL1/RKL2 and adaptive RKL1/RKL2, of
different sizes so that one packed launch spans problems of several shapes)
and requests the batch launches on their own (FP64, odd nx, masked storage,
adaptive SSP(10)4); a budget smaller than the whole mix makes admission wait
for memory to free up."""
import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I

from test_gpu_parity import pf  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

TOL = (1e-4, 1e-3, 1e-4, 1e-4)


def _mix(pf):
    R = []
    prob, u = I.circle(64, 18.0, W=2.5)
    R.append((prob, u, 32, 0, pf.FEULER, dict(dt_mult=0.9), 40))
    prob, u = I.multiphase_blobs(48, 34, 1, 5, seed=3, has_conc=1, n_alpha=2)
    R.append((prob, u, 32, 0, pf.RKL2, dict(tol=TOL), 30))
    R.append((prob, u, 32, 0, pf.RKL1, dict(dt_mult=6.0), 30))
    prob, u = I.multiphase_blobs(20, 18, 12, 6, seed=6, has_conc=1, n_alpha=1)
    R.append((prob, u, 32, 0, pf.RKL2, dict(dt_mult=12.0), 25))
    R.append((prob, u, 32, 0, pf.SSP2, dict(dt_mult=2.0), 25))
    prob, u = I.multiphase_blobs(32, 30, 8, 9, seed=8, has_conc=0, min_dist=6.0)
    R.append((prob, u, 32, 0, pf.RKL1, dict(tol=TOL), 30))
    prob, u = I.stefan(nx=128, ny=4, h=30.0, W=2.5)
    R.append((prob, u, 32, 0, pf.RKL2, dict(tol=TOL), 60))
    # launched on their own by the batch
    prob, u = I.multiphase_blobs(17, 13, 1, 4, seed=3, has_conc=1, n_alpha=1)
    R.append((prob, u, 64, 0, pf.RKL2, dict(tol=TOL), 30))                  # FP64
    R.append((prob, u, 32, 0, pf.FEULER, dict(dt_mult=0.9), 20))            # odd nx
    prob, u = I.multiphase_blobs(24, 20, 10, 7, seed=9, has_conc=0)
    R.append((prob, u, 32, pf.Simulation.OPT_MASKED, pf.RKL2, dict(tol=TOL), 25))   # masked
    R.append((prob, u, 32, 0, pf.SSP104, dict(tol=TOL), 25))                # SSP(10)4
    return R


def _alone(pf, prob, u, prec, opts, integ, kw, n):
    with pf.Simulation(prob, precision=prec, options=opts) as sim:
        sim.set_state(u)
        st = sim.step(integ, n * sim.dt_e(), **kw)
        return sim.get_state()[0], st


def test_batch_results_equal_the_requests_alone(pf):
    import torch
    mix = _mix(pf)
    ref = [_alone(pf, *m) for m in mix]
    stream = torch.cuda.Stream()
    total = sum(pf.footprint(m[0], m[2], m[3]) for m in mix)
    budget = int(0.6 * total)
    with pf.Batch(budget, stream=stream) as batch:
        waiting = list(range(len(mix)))
        running, results = {}, {}
        rounds = 0
        while waiting or running:
            while waiting:
                prob, u, prec, opts, integ, kw, n = mix[waiting[0]]
                sim = pf.Simulation(prob, precision=prec, stream=stream, options=opts)
                sim.set_state(u)
                slot = batch.admit(sim, integ, n * sim.dt_e(), **kw)
                if slot is None:
                    sim.close()
                    assert running                        # something must be holding the budget
                    break
                running[slot] = (waiting.pop(0), sim)
            batch.run(2)
            rounds += 1
            for slot in list(running):
                res = batch.result(slot)
                if res is not None:
                    k, sim = running.pop(slot)
                    results[k] = (res, sim.get_state())
                    sim.close()
    assert rounds > 3
    for k, ((status, st), (ub, tb)) in sorted(results.items()):
        ua, sa = ref[k]
        assert status == pf.PF_OK, k
        assert tb == sa["t"], k
        for key in ("rhs_evals", "steps_accepted", "steps_rejected"):
            assert st[key] == sa[key], (k, key)
        np.testing.assert_array_equal(ub, ua, err_msg="request %d" % k)
    assert len(results) == len(mix)


def test_batch_failure_is_per_request(pf):
    # a request whose state is not finite fails with PF_EUNSTABLE and keeps
    # its state; the request packed beside it is unaffected
    import torch
    prob, good = I.multiphase_blobs(48, 34, 1, 5, seed=3, has_conc=1, n_alpha=2)
    bad = good.copy()
    bad[prob.n_phases, 77] = np.nan
    ua, sa = _alone(pf, prob, good, 32, 0, pf.RKL2, dict(dt_mult=8.0), 40)
    stream = torch.cuda.Stream()
    with pf.Batch(1 << 34, stream=stream) as batch:
        sims = []
        for u in (good, bad):
            sim = pf.Simulation(prob, precision=32, stream=stream)
            sim.set_state(u)
            sims.append((batch.admit(sim, pf.RKL2, 40 * sim.dt_e(), dt_mult=8.0), sim))
        while batch.run(4):
            pass
        (sg, simg), (sb, simb) = sims
        status_g, st_g = batch.result(sg)
        status_b, st_b = batch.result(sb)
        ug, tg = simg.get_state()
        ub, tb = simb.get_state()
    assert status_g == pf.PF_OK and status_b == pf.PF_EUNSTABLE
    np.testing.assert_array_equal(ug, ua)
    assert tb == 0.0 and st_b["steps_accepted"] == 0
    assert np.isnan(ub).any()                         # its own last accepted state: the input


def test_batch_admission_rules(pf):
    import torch
    prob, u = I.circle(64, 18.0, W=2.5)
    fp = pf.footprint(prob, 32)
    stream = torch.cuda.Stream()
    with pf.Batch(fp + fp // 2, stream=stream) as batch:
        a = pf.Simulation(prob, precision=32, stream=stream)
        b = pf.Simulation(prob, precision=32, stream=stream)
        a.set_state(u)
        b.set_state(u)
        sa = batch.admit(a, pf.FEULER, 10 * a.dt_e(), dt_mult=0.9)
        assert sa is not None
        assert batch.admit(b, pf.FEULER, 10 * b.dt_e(), dt_mult=0.9) is None      # over budget
        with pytest.raises(pf.PfError):
            a.step(pf.FEULER, 20 * a.dt_e(), dt_mult=0.9)                        # owned by the batch
        with pytest.raises(pf.PfError):
            batch.admit(a, pf.FEULER, 10 * a.dt_e(), dt_mult=0.9)                # already admitted
        assert batch.result(sa) is None                                          # not run yet
        while batch.run(8):
            pass
        status, st = batch.result(sa)
        assert status == pf.PF_OK and st["steps_accepted"] == 12          # ceil(10 / 0.9) fixed steps
        assert batch.admit(b, pf.FEULER, 10 * b.dt_e(), dt_mult=0.9) is not None # budget freed
        while batch.run(8):
            pass
        a.close()
        b.close()


def test_torch_allocator_backs_the_handles(pf):
    import torch
    prob, u = I.multiphase_blobs(48, 34, 1, 5, seed=3, has_conc=1, n_alpha=2)
    ref, _ = _alone(pf, prob, u, 32, 0, pf.RKL2, dict(tol=TOL), 20)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    pf.use_torch_allocator(True)
    try:
        sim = pf.Simulation(prob, precision=32, stream=torch.cuda.Stream())
        during = torch.cuda.memory_allocated()
        assert during - before >= 5 * prob.nfields * prob.V * 4    # the five state vectors at least
        sim.set_state(u)
        sim.step(pf.RKL2, 20 * sim.dt_e(), tol=TOL)
        out, _ = sim.get_state()
        sim.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before            # all of it came back
    finally:
        pf.use_torch_allocator(False)
    np.testing.assert_array_equal(out, ref)
    with pf.Simulation(prob, precision=32) as sim:                  # default allocator again
        assert torch.cuda.memory_allocated() == before
