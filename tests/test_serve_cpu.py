"""Scheduling logic of the serving loop (no GPU): admission by footprint,
arrival order, budget never exceeded, oversize requests refused, every
request finished (continuous batching: freed memory is reused at once)."""
import threading
import time

import numpy as np

from paper_2601_16522_gb300.serve import Request, Server, summary


class FakeProb:
    def __init__(self, V):
        self.V = V


def make(n, seed=0, budget=100):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        r = Request(rid=i, prob=FakeProb(int(rng.integers(10, 1000))), u0=None, integ=0, t_end=1.0,
                    arrival=0.001 * i)
        r.fp = int(rng.integers(5, 60)) if i != 7 else budget + 1
        reqs.append(r)
    return reqs


def test_admission_respects_budget_and_order():
    budget = 100
    reqs = make(40, budget=budget)
    live = {"now": 0, "max": 0}
    lock = threading.Lock()
    order = []

    def runner(req, stream):
        with lock:
            live["now"] += req.fp
            live["max"] = max(live["max"], live["now"])
            order.append(req.rid)
        time.sleep(0.002 + 0.001 * (req.rid % 3))
        with lock:
            live["now"] -= req.fp
        return np.zeros(1), {"rhs_evals": 3}

    srv = Server(budget, workers=4, runner=runner, stream_factory=lambda: None, footprint=lambda r: r.fp)
    finished, makespan = srv.serve(reqs, realtime=True)
    assert len(finished) == len(reqs)
    assert live["max"] <= budget and srv.peak_used <= budget
    refused = [r for r in finished if r.error]
    assert [r.rid for r in refused] == [7]
    # admission follows arrival order (FIFO, no overtaking)
    assert order == sorted(order)
    s = summary(finished, makespan)
    assert s["completed"] == len(reqs) - 1 and s["rejected"] == 1
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_memory_freed_is_reused():
    # three requests of 60 with a budget of 100 run one at a time
    reqs = [Request(rid=i, prob=FakeProb(10), u0=None, integ=0, t_end=1.0, arrival=0.0) for i in range(3)]
    spans = []

    def runner(req, stream):
        t = time.perf_counter()
        time.sleep(0.01)
        spans.append((t, time.perf_counter()))
        return np.zeros(1), {"rhs_evals": 1}

    srv = Server(100, workers=3, runner=runner, stream_factory=lambda: None, footprint=lambda r: 60)
    finished, _ = srv.serve(reqs, realtime=False)
    assert len(finished) == 3 and all(r.error is None for r in finished)
    spans.sort()
    assert all(spans[i][1] <= spans[i + 1][0] + 1e-3 for i in range(2))


def test_failing_request_releases_its_memory():
    # A run that raises (the engine's PF_EINVAL on a list-capacity overflow,
    # say) is reported on that request; its memory and worker are released
    # and the requests behind it still run.
    reqs = [Request(rid=i, prob=FakeProb(10), u0=None, integ=0, t_end=1.0, arrival=0.0) for i in range(6)]

    def runner(req, stream):
        if req.rid == 2:
            raise RuntimeError("pf_step failed: invalid argument (status 1)")
        time.sleep(0.002)
        return np.zeros(1), {"rhs_evals": 1}

    srv = Server(100, workers=2, runner=runner, stream_factory=lambda: None, footprint=lambda r: 60)
    finished, makespan = srv.serve(reqs, realtime=False)
    assert len(finished) == 6
    bad = [r for r in finished if r.error]
    assert [r.rid for r in bad] == [2] and "status 1" in bad[0].error
    assert srv.used == 0 and srv.peak_used <= 100
    s = summary(finished, makespan)
    assert s["completed"] == 5 and s["rejected"] == 1


def test_cancellation_of_queued_and_running_requests():
    # Host-side cancellation: a request cancelled while it waits for memory
    # leaves without ever running; one cancelled while its (uninterruptible)
    # run is in progress finishes normally; the rest are unaffected.
    reqs = [Request(rid=i, prob=FakeProb(10), u0=None, integ=0, t_end=1.0, arrival=0.0) for i in range(5)]
    started = {}
    gate = threading.Event()
    ran = []

    def runner(req, stream):
        ran.append(req.rid)
        started[req.rid] = True
        if req.rid == 0:
            gate.wait(timeout=5.0)                 # holds the whole budget until released
        return np.zeros(1), {"rhs_evals": 1}

    srv = Server(100, workers=2, runner=runner, stream_factory=lambda: None, footprint=lambda r: 60)
    out = {}
    th = threading.Thread(target=lambda: out.update(res=srv.serve(reqs, realtime=False)))
    th.start()
    t0 = time.perf_counter()
    while 0 not in started and time.perf_counter() - t0 < 5.0:
        time.sleep(0.001)
    assert srv.cancel(0) is True                   # running: not interrupted
    assert srv.cancel(3) is True                   # queued behind request 0
    assert srv.cancel(99) is False                 # unknown
    gate.set()
    th.join(timeout=10.0)
    assert not th.is_alive()
    finished, makespan = out["res"]
    by = {r.rid: r for r in finished}
    assert len(finished) == 5
    assert by[0].error is None and by[0].result is not None
    assert by[3].error.startswith("cancelled before admission") and 3 not in ran
    assert all(by[i].error is None for i in (1, 2, 4))
    assert srv.used == 0
    s = summary(finished, makespan)
    assert s["completed"] == 4 and s["cancelled"] == 1 and s["rejected"] == 0
    assert srv.cancel(1) is False                  # finished


def test_poisson_stream_follows_its_recipe():
    # The served stream's recipe: Poisson arrivals (mean rate 50/s, seed 4),
    # 2D circles and Stefan strips (N = 2), 2D/3D Voronoi grain structures
    # with 2..32 phases in masked storage, the five integrators (SSP(10)4 and
    # the RKL schemes adaptive), each request
    # carrying its own state of the right shape; the same seed gives the same
    # stream.
    from paper_2601_16522_gb300 import serve
    a = serve.poisson_stream(30, rate=50.0, seed=4, sizes3d=(64,), device="cpu")
    b = serve.poisson_stream(30, rate=50.0, seed=4, sizes3d=(64,), device="cpu")
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0) and 0.1 < arr[-1] < 2.0        # ~30 / 50 s
    for r, s in zip(a, b):
        assert r.arrival == s.arrival and r.integ == s.integ and r.prob.name == s.prob.name
        assert np.array_equal(r.u0, s.u0)
    kinds = set()
    for r in a:
        p = r.prob
        assert r.u0.shape == (p.n_phases + p.has_conc, p.V)
        assert np.allclose(r.u0[:p.n_phases].sum(0), 1.0, atol=1e-12)
        assert r.integ in (0, 1, 2, 3, 4)
        assert (r.tol is not None) == (r.integ in (2, 3, 4))
        if p.name.startswith("grains"):
            kinds.add("grains")
            assert 2 <= p.n_phases <= 32 and r.options == 2
        else:
            kinds.add(p.name.rstrip("0123456789x"))
            assert p.n_phases == 2 and p.dim == 2 and r.options == 0
    assert kinds == {"grains", "circle", "stefan"}
