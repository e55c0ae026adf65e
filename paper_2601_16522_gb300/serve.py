"""Serving loops: continuous batching of simulations by device-memory footprint.

BatchServer drives the library's batch (pf_batch_*: one stream, one round of
steps at a time, the passes of FP32 dense problems packed into shared
launches).  Server below is the thread-per-request form:

Requests (a problem, an initial state, an integrator and an end time) arrive
over time.  The scheduler admits a waiting request as soon as its footprint
(pf_footprint) fits into the memory budget and a worker is free; an admitted
request gets its own handle on its own CUDA stream and a worker thread drives
it to its end time through the C ABI (ctypes releases the GIL during the
call), so the kernels of all resident requests overlap on the GPU.  When a
request finishes, its state is copied out, its handle and memory are
released, and the next waiting requests are admitted.  Every result is
computed by exactly the same passes as a stand-alone run, so a request's
result does not depend on what it was batched with.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import inputs as I
from . import pf


@dataclass
class Request:
    rid: int
    prob: I.Problem
    u0: np.ndarray                  # (N + K, V) float64
    integ: int
    t_end: float
    tol: Optional[tuple] = None     # adaptive when set, else fixed dt_mult
    dt_mult: float = 0.0
    precision: int = 32
    options: int = 0                # pf_params.options (e.g. masked storage)
    arrival: float = 0.0            # seconds after the start of the stream
    # filled in by the server
    admitted: float = float("nan")
    finished: float = float("nan")
    result: Optional[np.ndarray] = None
    stats: Optional[dict] = None
    error: Optional[str] = None
    cancelled: bool = False         # set by Server.cancel

    @property
    def footprint(self):
        return pf.footprint(self.prob, self.precision, self.options)

    @property
    def latency(self):
        return self.finished - self.arrival

    def describe(self):
        p = self.prob
        dims = [getattr(p, k, None) for k in ("nx", "ny", "nz")][:2 if getattr(p, "dim", 3) == 2 else 3]
        size = "x".join(str(v) for v in dims) if None not in dims else "V=%s" % getattr(p, "V", "?")
        return "request %d: %s %s, %s phases%s, integrator %d, %s" % (
            self.rid, getattr(p, "name", "") or "problem", size, getattr(p, "n_phases", "?"),
            " + c" if getattr(p, "has_conc", 0) else "", self.integ,
            "tol %s" % (self.tol,) if self.tol is not None else "dt_mult %g" % self.dt_mult)


def run_alone(req: Request, stream=None):
    """Run one request by itself (reference for the batching invariance)."""
    import torch
    stream = stream or torch.cuda.Stream()
    with pf.Simulation(req.prob, precision=req.precision, stream=stream, options=req.options) as sim:
        sim.set_state(req.u0)
        st = _advance(sim, req)
        out, _ = sim.get_state()
    return out, st


def _advance(sim, req):
    if req.tol is not None:
        return sim.step(req.integ, req.t_end, tol=req.tol)
    return sim.step(req.integ, req.t_end, dt_mult=req.dt_mult)


class Server:
    """Admit by footprint, run on worker threads with one stream each.

    runner(request, stream) -> (state, stats) does the work (default: the C
    ABI on the GPU); stream_factory() makes one stream per worker; footprint
    (request) -> bytes.  Tests of the scheduling logic replace all three."""

    def __init__(self, mem_budget_bytes: int, workers: int = 8, runner=None, stream_factory=None,
                 footprint=None):
        self.budget = int(mem_budget_bytes)
        self.workers = int(workers)
        self.used = 0
        self.peak_used = 0
        self.lock = threading.Condition()
        self.runner = runner or run_alone
        self.stream_factory = stream_factory
        self.footprint = footprint or (lambda r: r.footprint)
        self._by_rid = {}

    def cancel(self, rid):
        """Cancel request `rid` (from any thread).  A request that has not
        been admitted leaves without using memory or a worker; one whose run
        has not started yet releases them at once; an engine call that is
        already running is not interrupted and its result is kept.  Returns
        whether the request was still unfinished."""
        with self.lock:
            r = self._by_rid.get(rid)
            if r is None or r.finished == r.finished:          # unknown or finished (not NaN)
                return False
            r.cancelled = True
            self.lock.notify_all()
            return True

    def serve(self, requests, realtime=True):
        """Feed the requests at their arrival times (realtime) or all at once;
        returns the finished requests and the makespan in seconds."""
        if self.stream_factory is None:
            import torch
            dev = torch.cuda.current_device()
            make_stream = lambda: torch.cuda.Stream(device=dev)       # noqa: E731
            set_dev = lambda: torch.cuda.set_device(dev)               # noqa: E731
        else:
            make_stream = self.stream_factory
            set_dev = lambda: None                                      # noqa: E731
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        with self.lock:
            self._by_rid = {r.rid: r for r in pending}
        fp = {r.rid: self.footprint(r) for r in pending}
        for r in pending:
            if fp[r.rid] > self.budget:
                r.error = "footprint %d B exceeds the memory budget %d B" % (fp[r.rid], self.budget)
        waiting = []          # arrived, not admitted (FIFO by arrival)
        running = []
        streams = [make_stream() for _ in range(self.workers)]
        free_streams = list(range(self.workers))
        t0 = time.perf_counter()
        nxt = 0
        finished = []

        def work(req, sidx):
            try:
                if req.cancelled:
                    req.error = "cancelled before its run started (%s)" % req.describe()
                    return
                set_dev()
                out, st = self.runner(req, streams[sidx])
                req.result, req.stats = out, st
            except Exception as exc:                  # reported per request
                req.error = "%s (%s)" % (exc, req.describe())
            finally:                                  # memory and worker come back whatever happened
                req.finished = time.perf_counter() - t0
                with self.lock:
                    self.used -= fp[req.rid]
                    free_streams.append(sidx)
                    finished.append(req)
                    self.lock.notify_all()

        while nxt < len(pending) or waiting or running:
            now = time.perf_counter() - t0
            while nxt < len(pending) and (not realtime or pending[nxt].arrival <= now):
                r = pending[nxt]
                nxt += 1
                if r.cancelled and not r.error:
                    r.error = "cancelled before admission (%s)" % r.describe()
                if r.error:
                    r.finished = now
                    finished.append(r)
                else:
                    waiting.append(r)
            with self.lock:
                # requests cancelled while queued leave without memory or a worker
                for r in [w for w in waiting if w.cancelled]:
                    waiting.remove(r)
                    r.error = "cancelled before admission (%s)" % r.describe()
                    r.finished = time.perf_counter() - t0
                    finished.append(r)
                # admit in arrival order while memory and a worker are available
                while waiting and free_streams and self.used + fp[waiting[0].rid] <= self.budget:
                    r = waiting.pop(0)
                    self.used += fp[r.rid]
                    self.peak_used = max(self.peak_used, self.used)
                    r.admitted = time.perf_counter() - t0
                    sidx = free_streams.pop(0)
                    th = threading.Thread(target=work, args=(r, sidx), daemon=True)
                    running.append(th)
                    th.start()
                running = [th for th in running if th.is_alive()]
                if nxt < len(pending):
                    wait = max(0.0, pending[nxt].arrival - (time.perf_counter() - t0)) if realtime else 0.0
                    self.lock.wait(timeout=min(wait, 0.05) if wait > 0 else 0.001)
                elif running or waiting:
                    self.lock.wait(timeout=0.05)
        makespan = time.perf_counter() - t0
        return finished, makespan


class BatchServer:
    """Continuous batching through the library's batch (pf_batch_*).

    Requests are sorted into lanes by the work of one step (cells times
    fields); every lane is one pf.Batch on its own CUDA stream, driven by its
    own thread (ctypes releases the GIL while the library runs), so lanes
    overlap on the GPU and a small request is not held back by the rounds of
    a large one.  Within a lane the batch advances all admitted requests a
    round at a time (one step or attempt each, the passes of FP32 dense
    problems packed into shared launches, one transfer of error norms and
    flags per round).  Arrivals are admitted, in arrival order, while the
    server's memory budget allows; finished requests leave with their state
    and statistics.  A result equals the request run alone (the batch keeps
    pf_step's bookkeeping).

    lane_bounds: upper bounds of cells x fields of all lanes but the last;
    rounds: rounds per batch call between admission checks; lane_cap: the
    most requests a lane runs at a time (arrivals queue per lane in arrival
    order, so that under load the early requests finish first instead of
    every request sharing the GPU with all later ones)."""

    def __init__(self, mem_budget_bytes: int, rounds: int = 4, lane_bounds=(1 << 20, 1 << 24), lane_cap=64):
        self.budget = int(mem_budget_bytes)
        self.rounds = int(rounds)
        self.lane_bounds = tuple(lane_bounds)
        self.lane_cap = int(lane_cap)
        self.peak_used = 0

    def _lane(self, r):
        w = r.prob.V * (r.prob.n_phases + r.prob.has_conc)
        for k, b in enumerate(self.lane_bounds):
            if w < b:
                return k
        return len(self.lane_bounds)

    def serve(self, requests, realtime=True):
        import torch
        dev = torch.cuda.current_device()
        nl = len(self.lane_bounds) + 1
        streams = [torch.cuda.Stream(device=dev) for _ in range(nl)]
        batches = [pf.Batch(self.budget, stream=st) for st in streams]
        locks = [threading.Lock() for _ in range(nl)]
        running = [dict() for _ in range(nl)]          # slot -> (request, simulation)
        cv = threading.Condition()
        state = {"used": 0, "stop": False}
        finished = []
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        fp = {r.rid: r.footprint for r in pending}
        t0 = time.perf_counter()

        def drive(k):
            torch.cuda.set_device(dev)
            while True:
                with cv:
                    while not running[k] and not state["stop"]:
                        cv.wait(0.05)
                    if state["stop"] and not running[k]:
                        return
                with locks[k]:
                    batches[k].run(self.rounds)
                    done = []
                    for slot in list(running[k]):
                        res = batches[k].result(slot)
                        if res is None:
                            continue
                        r, sim = running[k].pop(slot)
                        status, st = res
                        if status == pf.PF_OK:
                            r.result, _ = sim.get_state()
                            r.stats = st
                        else:
                            r.error = "status %d (%s)" % (status, r.describe())
                        sim.close()
                        r.finished = time.perf_counter() - t0
                        done.append(r)
                if done:
                    with cv:
                        for r in done:
                            state["used"] -= fp[r.rid]
                            finished.append(r)
                        cv.notify_all()

        threads = [threading.Thread(target=drive, args=(k,), daemon=True) for k in range(nl)]
        for th in threads:
            th.start()
        waiting = [[] for _ in range(nl)]              # per lane, arrival order
        nxt = 0
        try:
            while True:
                now = time.perf_counter() - t0
                while nxt < len(pending) and (not realtime or pending[nxt].arrival <= now):
                    r = pending[nxt]
                    nxt += 1
                    if fp[r.rid] > self.budget:
                        r.error = "footprint %d B exceeds the memory budget %d B" % (fp[r.rid], self.budget)
                        r.finished = now
                        with cv:
                            finished.append(r)
                    else:
                        waiting[self._lane(r)].append(r)
                # admit in arrival order per lane while the lane has room and the budget allows
                for k in range(nl):
                    while waiting[k]:
                        r = waiting[k][0]
                        with cv:
                            if state["used"] + fp[r.rid] > self.budget or len(running[k]) >= self.lane_cap:
                                break
                            state["used"] += fp[r.rid]
                            self.peak_used = max(self.peak_used, state["used"])
                        waiting[k].pop(0)
                        err = None
                        with locks[k]:
                            sim = pf.Simulation(r.prob, precision=r.precision, stream=streams[k], options=r.options)
                            try:
                                sim.set_state(r.u0)
                                slot = batches[k].admit(sim, r.integ, r.t_end, tol=r.tol, dt_mult=r.dt_mult)
                                if slot is None:
                                    err = "not admitted by the batch (%s)" % r.describe()
                            except Exception as exc:
                                err = "%s (%s)" % (exc, r.describe())
                            if err is None:
                                r.admitted = time.perf_counter() - t0
                                running[k][slot] = (r, sim)
                            else:
                                sim.close()
                        with cv:
                            if err is not None:
                                r.error = err
                                r.finished = time.perf_counter() - t0
                                state["used"] -= fp[r.rid]
                                finished.append(r)
                            cv.notify_all()
                with cv:
                    if nxt >= len(pending) and not any(waiting) and len(finished) == len(pending):
                        break
                    wait = 0.002
                    if nxt < len(pending) and realtime:
                        wait = max(0.0005, min(0.01, pending[nxt].arrival - (time.perf_counter() - t0)))
                    cv.wait(wait)
        finally:
            with cv:
                state["stop"] = True
                cv.notify_all()
            for th in threads:
                th.join()
            for b in batches:
                b.close()
        return finished, time.perf_counter() - t0


def poisson_stream(n, rate=50.0, seed=4, sizes2d=(64, 128, 256, 512, 1024), sizes3d=(64, 96, 128, 192),
                   phases=(2, 3, 8, 16, 32), steps=100, device="cuda", masked_grains=True):
    """Seeded mixed stream shaped like the paper's benchmarks: shrinking
    circles and Stefan strips (2D, N = 2) and Voronoi grain structures (2D/3D,
    N up to 32, in masked storage unless masked_grains is False); integrators
    (FE, SSP(5)2, RKL1, RKL2, adaptive SSP(10)4) and tolerances drawn
    uniformly.  Each request runs for `steps` stable Euler steps of
    simulated time."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        kind = rng.integers(0, 3)
        if kind == 0:
            nn = int(rng.choice(sizes2d))
            prob, u = I.circle(nn, 0.3 * nn, W=2.5)
        elif kind == 1:
            nn = int(rng.choice(sizes2d))
            prob, u = I.stefan(nx=max(64, nn), ny=max(8, nn // 4), h=0.2 * max(64, nn), W=2.5)
        else:
            dim = int(rng.integers(2, 4))
            nn = int(rng.choice(sizes3d if dim == 3 else sizes2d[:3]))
            N = int(rng.choice(phases))
            N = max(2, min(N, max(2, (nn // 16) ** dim)))
            prob, u = I.grains_device(n=nn, n_grains=N, min_dist=0.5 * nn / N ** (1.0 / dim),
                                      seed=int(rng.integers(1 << 30)), dim=dim, dx=1.0, W_cells=2.5, M=1.0,
                                      device=device)
            u = u.cpu().numpy()
        integ = int(rng.choice([pf.FEULER, pf.RKL1, pf.RKL2, pf.SSP2, pf.SSP104]))
        a_phi = float(rng.choice([1e-2, 1e-3, 1e-4]))
        # grain structures run in masked storage (only occupied phases are loaded)
        opts = pf.Simulation.OPT_MASKED if (kind == 2 and masked_grains) else 0
        req = Request(rid=rid, prob=prob, u0=u, integ=integ, t_end=0.0, arrival=t, options=opts)
        if integ in (pf.RKL1, pf.RKL2, pf.SSP104):
            req.tol = (1e-4, a_phi, 1e-4, 1e-4)
        else:
            req.dt_mult = 0.9 if integ == pf.FEULER else 2.0
        req.steps = steps
        reqs.append(req)
    return reqs


def finalize_end_times(reqs):
    """Set each request's end time to `steps` stable Euler steps (needs dt_e)."""
    for r in reqs:
        with pf.Simulation(r.prob, precision=r.precision) as sim:
            r.t_end = r.steps * sim.dt_e()
    return reqs


def summary(finished, makespan):
    ok = [r for r in finished if r.error is None]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    cells = sum(r.prob.V * r.stats["rhs_evals"] for r in ok)
    cancelled = [r for r in finished if r.error is not None and r.cancelled]
    errors = [r.error for r in finished if r.error is not None and not r.cancelled]
    return {"requests": len(finished), "completed": len(ok), "rejected": len(errors),
            "cancelled": len(cancelled), "errors": errors[:5],
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "makespan_s": makespan, "gcell_updates_per_s": cells / makespan / 1e9}
