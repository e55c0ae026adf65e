"""Serving on the GPU: a request's result is the same alone and in a mix of
concurrently running requests (bit for bit: every request runs the same
passes on its own stream and buffers; reductions have a fixed order)."""
import numpy as np
import pytest

from paper_2601_16522_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16522_gb300 import build
    build.build()
    from paper_2601_16522_gb300 import pf, serve
    return torch, pf, serve


def requests(pf, serve):
    reqs = []
    p, u = I.circle(96, 30.0, W=2.5)
    reqs.append(serve.Request(0, p, u, pf.RKL2, 0.0, tol=(1e-4, 1e-2, 1e-4, 1e-4), precision=32))
    p, u = I.stefan(nx=256, ny=16, h=60.0, W=2.5)
    reqs.append(serve.Request(1, p, u, pf.FEULER, 0.0, dt_mult=0.9, precision=64))
    p, u = I.multiphase_blobs(40, 36, 20, 6, seed=3, has_conc=1, n_alpha=1)
    reqs.append(serve.Request(2, p, u, pf.RKL1, 0.0, tol=(1e-4, 1e-3, 1e-4, 1e-4), precision=32))
    p, u = I.grains(n=48, n_grains=8, min_dist=14.0, seed=5, dim=3, dx=1.0, W_cells=2.5, M=1.0)
    reqs.append(serve.Request(3, p, u, pf.SSP2, 0.0, dt_mult=2.0, precision=32))
    p, u = I.multiphase_blobs(64, 32, 16, 12, seed=21, W=2.0, min_dist=9.0)
    reqs.append(serve.Request(4, p, u, pf.RKL2, 0.0, dt_mult=20.0, precision=32))
    p, u = I.circle(64, 20.0, W=2.5)
    reqs.append(serve.Request(5, p, u, pf.SSP104, 0.0, tol=(1e-4, 1e-2, 1e-4, 1e-4), precision=64))
    for r in reqs:
        r.steps = 60
    serve.finalize_end_times(reqs)
    for k, r in enumerate(reqs):
        r.arrival = 0.002 * k
    return reqs


def test_alone_equals_mixed(env):
    torch, pf, serve = env
    alone = {}
    for r in requests(pf, serve):
        out, st = serve.run_alone(r)
        alone[r.rid] = (out, st["rhs_evals"])
    reqs = requests(pf, serve)
    srv = serve.Server(mem_budget_bytes=8 << 30, workers=4)
    finished, makespan = srv.serve(reqs, realtime=True)
    assert len(finished) == len(reqs)
    for r in finished:
        assert r.error is None, r.error
        np.testing.assert_array_equal(r.result, alone[r.rid][0])
        assert r.stats["rhs_evals"] == alone[r.rid][1]
    s = serve.summary(finished, makespan)
    assert s["completed"] == len(reqs) and s["gcell_updates_per_s"] > 0


def test_tight_budget_still_completes(env):
    torch, pf, serve = env
    reqs = requests(pf, serve)
    biggest = max(pf.footprint(r.prob, r.precision) for r in reqs)
    srv = serve.Server(mem_budget_bytes=biggest, workers=4)
    finished, _ = srv.serve(reqs, realtime=False)
    assert all(r.error is None for r in finished) and len(finished) == len(reqs)
    assert srv.peak_used <= biggest


@pytest.mark.parametrize("bounds", [(1 << 20, 1 << 24), ()], ids=["three-lanes", "one-lane"])
def test_batch_server_alone_equals_mixed(env, bounds):
    # the batch server (pf_batch_*, packed launches, lanes on their own
    # streams and threads) gives every request the result it has alone
    torch, pf, serve = env
    alone = {}
    for r in requests(pf, serve):
        out, st = serve.run_alone(r)
        alone[r.rid] = (out, st["rhs_evals"])
    reqs = requests(pf, serve)
    srv = serve.BatchServer(mem_budget_bytes=8 << 30, rounds=3, lane_bounds=bounds)
    finished, makespan = srv.serve(reqs, realtime=True)
    assert len(finished) == len(reqs)
    for r in finished:
        assert r.error is None, r.error
        np.testing.assert_array_equal(r.result, alone[r.rid][0])
        assert r.stats["rhs_evals"] == alone[r.rid][1]
    # a budget that holds only the largest request at a time
    reqs = requests(pf, serve)
    biggest = max(pf.footprint(r.prob, r.precision) for r in reqs)
    srv = serve.BatchServer(mem_budget_bytes=biggest, rounds=2, lane_bounds=bounds)
    finished, _ = srv.serve(reqs, realtime=False)
    assert all(r.error is None for r in finished) and len(finished) == len(reqs)
    assert srv.peak_used <= biggest
