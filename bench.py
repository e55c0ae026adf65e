#!/usr/bin/env python
"""Benchmark: GCell-updates/s of the explicit phase-field step on one GB300.

Workload (default ``grains256``): 3D grain growth, 256^3 periodic cells, 32
grains from a seeded periodic Voronoi tessellation with diffuse boundaries,
dense N = 32 phase storage in FP32 (FP64 time, coefficients and reductions),
paper units dx = 0.005, W = 2.5 dx, M = 5e-3, gamma = 1.  One step = one
attempted adaptive RKL2 step (Sec. 3.2-3.3): s fused stage passes (RHS, stage
combination, simplex projection, first-stage fix), the error sweep with the
weighted norm, and the PID controller.  Every state vector (2.1 GB) is larger
than L2, so no flush is needed between steps.

value = cells x RHS sweeps / device time (max over ranks, summed over ranks),
e2e   = the same through the C ABI with host buffers (pinned) copied in and out
        every step.

``--impl reference`` times the CPU oracle (the only reference this method has)
on a bounded sample of the same workload and prints the same line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TOL = (1e-4, 1e-2, 1e-4, 1e-3)          # r_phi, a_phi, r_c, a_c (Sec. 5.3 runs)
METRIC = "GCell-updates/s"
UNIT = "GCell/s"


def workload_problem(name, device):
    from paper_2601_16522_gb300 import inputs as I
    if name == "grains256":
        prob, u = I.grains_device(n=256, n_grains=32, min_dist=40.0, seed=2, dim=3, device=device)
        return prob, u, 32
    if name == "grains128":
        prob, u = I.grains_device(n=128, n_grains=32, min_dist=20.0, seed=2, dim=3, device=device)
        return prob, u, 32
    if name == "sinter320":
        prob, u = I.sintering_device(n=320, n_grains=64, seed=3, device=device)
        return prob, u, 32
    if name == "sinter160":
        prob, u = I.sintering_device(n=160, n_grains=64, seed=3, device=device)
        return prob, u, 32
    raise SystemExit("unknown workload %s" % name)


# algorithmic vectors moved per pass kind (reads + writes of whole state vectors)
PASS_VECTORS = {"rkl2": 5, "rkl1": 3, "sts_first": 3, "sts_err": 3, "euler": 2, "ssp": 2, "rhs": 1}
# DRAM bytes (read + write) per cell of one RKL2 stage pass (two-cell kernel,
# 32-phase FP32 state) from an ncu capture of that launch at full size
# (256^3: 8.822 GB read + 2.148 GB written in the second RKL2 pass of a step;
# the algorithmic 640 B/cell is 10.74 GB)
RKL2_TRAFFIC_PER_CELL = {"grains256": (8821829632 + 2148446464) / 16777216}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def kernel_name(prob, prec, variant):
    """Which stage kernel the library dispatches for this problem's RKL2
    passes (variant: the kernel variant the handle uses)."""
    K = prob.has_conc
    if prec == 64:
        return "cell_kernel<double,%d,%d,generic>" % (prob.dim, K)
    if prob.n_phases > 32:
        return "big_kernel<%d,%d,sig>" % (prob.dim, K)
    if variant == "tma" and prob.dim == 3 and prob.n_phases > 4:
        return "tma_kernel<%d,sig>" % K
    if variant == "two_cell" and prob.nx % 2 == 0:
        return "vec_kernel<%d,%d,sig> + wide_fix_kernel" % (prob.dim, K)
    return "fast_kernel<%d,%d,sig,%d>" % (prob.dim, K, 4 if prob.n_phases <= 4 else 32)


def max_over_ranks(x, world, device=None):
    """Maximum of a host scalar over the ranks (the timing rule for N > 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "gloo":
        device = None
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(cells, sweeps_per_rank, ms_max, world):
    """Whole-job GCell-updates/s: every rank runs its own replica of the same
    workload (weak scaling), so the job updates world x cells x sweeps cells
    in the slowest rank's time."""
    return world * cells * sweeps_per_rank / (ms_max * 1e-3) / 1e9


def oracle_configs():
    """The CPU oracle on the configurations beside the GPU runs: the
    shrinking circle (128^2, 2000 FE steps of 0.9 dt_e, FP64) in full, the
    Stefan strip (1024 x 256) for a
    fixed number of forward Euler steps (the Stefan count extrapolated to
    its run length, t = 43e3); the sintering recipe (65 phases + c) on a
    48^3 box; OpenMP on all host cores, and one thread on a tenth of the
    circle run."""
    from oracle import ref
    from paper_2601_16522_gb300 import inputs as I
    cores = os.cpu_count()
    out = {"cores": cores}

    def fe(prob, u, n_steps):
        o = ref.Oracle(prob)
        dte = o.dt_e()
        t0 = time.perf_counter()
        st, _, t, _ = o.run(ref.FEULER, u, 0.0, n_steps * 0.9 * dte, dt_mult=0.9)
        el = time.perf_counter() - t0
        return el, dte

    ref.set_openmp(True)
    try:
        prob, u = I.circle(128, 40.0)
        el, dte = fe(prob, u, 2000)
        out["circle128_fe64_full"] = {"steps": 2000, "wall_s": el, "gcell_updates_per_s": prob.V * 2000 / el / 1e9}
        prob, u = I.stefan(nx=1024, ny=256, h=200.0)
        el, dte = fe(prob, u, 20)
        n_full = math.ceil(43e3 / (0.9 * dte))
        out["stefan1024x256_fe64"] = {"steps_timed": 20, "wall_s": el, "gcell_updates_per_s": prob.V * 20 / el / 1e9,
                                      "steps_to_t43e3": n_full, "estimated_wall_s_to_t43e3": el / 20 * n_full}
        # the sintering recipe (64 grains + pore phase + c) on a 48^3 box
        sp, su = I.sintering_device(n=48, n_grains=64, seed=3, device="cpu")
        el, dte = fe(sp, su.numpy(), 2)
        out["sinter_recipe48_fe64"] = {"steps_timed": 2, "cells": sp.V, "phases": sp.n_phases, "wall_s": el,
                                       "gcell_updates_per_s": sp.V * 2 / el / 1e9}
    finally:
        ref.set_openmp(False)
    prob, u = I.circle(128, 40.0)
    el, dte = fe(prob, u, 200)
    out["circle128_fe64_single_thread"] = {"steps": 200, "wall_s": el, "gcell_updates_per_s": prob.V * 200 / el / 1e9}
    return out


def oracle_sample(u_host_sub, prob_sub, s=5):
    """Time the CPU oracle on one RKL2 step (s stages + error sweep) of a sub-box."""
    from oracle import ref
    o = ref.Oracle(prob_sub)
    dte = o.dt_e()
    dt = 0.9 * dte * ((s * s + s - 2) / 4.0) * 0.999
    t0 = time.perf_counter()
    _, e, _ = o.step_error(ref.RKL2, dt, s, u_host_sub, TOL)
    el = time.perf_counter() - t0
    sweeps = s + 1
    return prob_sub.V * sweeps / el / 1e9, el, sweeps


def sub_box(prob, u_dev, m):
    """Periodic m^3 sub-box (corner at the origin) of a 3D state, on the host."""
    import numpy as np
    n = prob.nx
    N = prob.n_phases
    NF = u_dev.shape[0]
    u3 = u_dev.reshape(NF, n, n, n)[:, :m, :m, :m].contiguous().cpu().numpy().reshape(NF, -1)
    sub = prob.with_(nx=m, ny=m, nz=m, name=prob.name + "_sub%d" % m)
    return sub, np.ascontiguousarray(u3)


def reference_sub_box(name, m):
    """The corner m^3 block of the workload's state, generated on the host only."""
    from paper_2601_16522_gb300 import inputs as I
    if name.startswith("sinter"):
        n = 320 if name == "sinter320" else 160
        prob, u = I.sintering_device(n=n, n_grains=64, seed=3, device="cpu")
        sub, us = sub_box(prob, u, m)
        return sub, us
    kw = dict(n=256, n_grains=32, min_dist=40.0) if name == "grains256" else dict(n=128, n_grains=32, min_dist=20.0)
    prob, u = I.grains_device(seed=2, dim=3, device="cpu", region=m, **kw)
    return prob.with_(nx=m, ny=m, nz=m, name=prob.name + "_sub%d" % m), u.numpy()


def run_reference(args, world, rank):
    """CPU oracle arm: each step is one oracle RKL2 step on a bounded sub-box."""
    if rank != 0:
        return
    m = 40
    sub, us = reference_sub_box(args.workload, m)
    vals = []
    tot_el, tot_cells = 0.0, 0.0
    for k in range(args.warmup + args.steps):
        v, el, sweeps = oracle_sample(us, sub)
        if k >= args.warmup:
            tot_el += el
            tot_cells += sub.V * sweeps
    value = tot_cells / tot_el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + " (oracle on a %d^3 periodic sub-box)" % m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one RKL2 step (s=5) + error sweep on a %d^3 sub-box of the same 32-phase state" % m},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# time to solution at fixed error (2D sharp-interface benchmarks)
# ---------------------------------------------------------------------------

def _area_rate_error(ts, areas, M=1.0, gamma=1.0):
    """|mean dA/dt + 2 pi M gamma| over t > 0, dA/dt by 2nd-order FD of the
    output series (Sec. 5.2.1); returned relative to 2 pi M gamma."""
    import numpy as np
    dA = np.gradient(np.asarray(areas), np.asarray(ts))[1:]
    exact = 2.0 * np.pi * M * gamma
    return abs(dA.mean() + exact) / exact


def _front(liquid_row):
    """x of phi_liquid = 0.5 by a cubic through the 4 nearest cell centres (Sec. 5.2.2)."""
    import numpy as np
    j = int(np.argmax(liquid_row >= 0.5))
    j = min(max(j, 2), len(liquid_row) - 2)
    xs = np.arange(j - 2, j + 2) + 0.5
    r = np.roots(np.polyfit(xs, liquid_row[j - 2:j + 2] - 0.5, 3))
    r = r[np.isreal(r)].real
    r = r[(r >= xs[0]) & (r <= xs[-1])]
    return float(r[0]) if len(r) else float(j)


def time_to_solution(pf, torch):
    """The shrinking circle (128^2, 2000 x 0.9 dt_e): wall time of each
    integrator/precision to t_end with outputs at exact times, and its error
    against the sharp-interface area law; FP64 forward Euler at 0.9 dt_e sets
    the target error.  (The Stefan strip is the stefan_sweep section.)"""
    import numpy as np
    from paper_2601_16522_gb300 import inputs as I
    res = {}
    # -- shrinking circle, 128^2, W = 5/pi, 2000 FE steps of 0.9 dt_e ----------
    prob, u = I.circle(128, 40.0)
    dloop = pf.Simulation.STEP_DEVICE_LOOP
    variants = [("feuler", 64, dict(dt_mult=0.9)), ("feuler", 32, dict(dt_mult=0.9)),
                ("rkl2", 32, dict(tol=(1e-4, 1e-2, 1e-4, 1e-4))), ("rkl2", 64, dict(tol=(1e-4, 1e-2, 1e-4, 1e-4))),
                ("rkl1", 32, dict(tol=(1e-4, 1e-2, 1e-4, 1e-4))),
                ("rkl2", 32, dict(tol=(1e-4, 1e-2, 1e-4, 1e-4), flags=dloop))]
    out = []
    stream = torch.cuda.Stream()
    for name, prec, kw in variants:
        sim = pf.Simulation(prob, precision=prec, stream=stream)
        sim.set_state(u)
        dte = sim.dt_e()
        t_end = 2000 * 0.9 * dte
        times = np.linspace(0.0, t_end, 41)
        integ = {"feuler": pf.FEULER, "rkl2": pf.RKL2, "rkl1": pf.RKL1}[name]
        areas = [sim.reduce()[1][1]]
        evals = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for tk in times[1:]:
            evals += sim.step(integ, float(tk), **kw)["rhs_evals"]
            areas.append(sim.reduce()[1][1])
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out.append({"integrator": name + ("-device-loop" if kw.get("flags") else ""), "precision": prec,
                    "wall_ms": 1e3 * el, "rhs_evals": evals, "rel_error": _area_rate_error(times, areas)})
        sim.close()
    res["circle128"] = {"t_end": "2000 x 0.9 dt_e", "error": "|<dA/dt> + 2 pi M gamma| / (2 pi M gamma)",
                        "variants": out}
    # speedups over FP64 FE among variants whose error is within 1.05x of its error
    for k, r in res.items():
        ref = [v for v in r["variants"] if v["integrator"] == "feuler" and v["precision"] == 64][0]
        r["target_error"] = ref["rel_error"]
        ok = [v for v in r["variants"] if v["rel_error"] <= 1.05 * ref["rel_error"] + 1e-12]
        best = min(ok, key=lambda v: v["wall_ms"])
        r["fastest_at_target"] = {"integrator": best["integrator"], "precision": best["precision"],
                                  "speedup_vs_fe64": ref["wall_ms"] / best["wall_ms"]}
    return res


def served_stream(pf, torch, n_requests, rate=50.0):
    """Poisson stream of mixed simulations through the continuous-batching
    server on the library's batch (pf_batch_*: one stream, a round of steps
    at a time, FP32 dense passes packed into shared launches); p50/p99
    latency and aggregate GCell-updates/s."""
    from paper_2601_16522_gb300 import serve
    reqs = serve.poisson_stream(n_requests, rate=rate, seed=4, sizes2d=(64, 128, 256, 512, 1024),
                                sizes3d=(64, 96, 128, 192), steps=100, masked_grains=True)
    serve.finalize_end_times(reqs)
    free, total = torch.cuda.mem_get_info()
    srv = serve.BatchServer(mem_budget_bytes=int(0.5 * free), rounds=4)
    lanes = "lanes by cells x fields < 2^20, < 2^24, larger (one batch, stream and thread each)"
    finished, makespan = srv.serve(reqs, realtime=True)
    s = serve.summary(finished, makespan)
    s.update({"arrival_rate_per_s": rate, "server": "batch (pf_batch_*), 4 rounds per call, " + lanes,
              "mem_budget_bytes": srv.budget, "peak_admitted_bytes": srv.peak_used,
              "mix": "circles, Stefan strips (2D 64^2..1024^2), 2D/3D Voronoi grains (N 2..32, 3D 64^3..192^3, "
                     "masked storage), FE/SSP(5)2 fixed and RKL1/RKL2/SSP(10)4 adaptive, FP32, "
                     "100 stable-Euler steps of simulated time each"})
    return s


def fp64_fe_pass(pf, torch, dev, stream):
    """Roofline of the FP64 forward Euler pass (the baseline of the
    time-to-solution comparisons) on the 256^3 x 32 grain workload: 2 x 32
    FP64 values per cell (read and write), timed over 3 passes."""
    prob, u, _ = workload_problem("grains256", dev)
    sim = pf.Simulation(prob, precision=64, stream=stream)
    sim.set_state(u)
    dte = sim.dt_e()
    sim.step(pf.FEULER, 0.9 * dte, dt_mult=0.9)
    sim.profile(1)
    sim.step(pf.FEULER, 4 * 0.9 * dte, dt_mult=0.9, flags=pf.Simulation.STEP_NO_GRAPH)
    prof = sim.profile(0)
    sim.close()
    ms, n = prof["euler"]
    nbytes = 2 * prob.n_phases * 8 * prob.V
    peak = _peak_gbs()
    ach = nbytes / (ms / n * 1e-3) / 1e9
    return {"workload": prob.name, "pass_ms": ms / n, "bytes_per_launch": nbytes, "achieved_gbs": ach,
            "frac_of_measured_peak": ach / peak, "kernel": "cell_kernel<double,3,0,generic> (--fmad=false)"}


def kernel_families(pf, torch, dev, stream):
    """The stage-pass kernel of every storage form, precision and projection
    on one workload (128^3 cells x 32 grains, vectors of 268 MB > L2): per
    launch time of the pass kind that dominates each run, its algorithmic
    bytes (state vectors read + written, dense-equivalent for masked storage)
    and their rate against the measured copy bandwidth; and the energy
    functional's pass (one vector read)."""
    prob, u, _ = workload_problem("grains128", dev)
    V, N = prob.V, prob.n_phases
    peak = _peak_gbs()
    O = pf.Simulation
    runs = [("rkl2 two-cell FP32", 32, 0, prob, pf.RKL2, "rkl2", 5),
            ("rkl2 one-cell FP32", 32, O.OPT_ONE_CELL, prob, pf.RKL2, "rkl2", 5),
            ("rkl2 masked FP32 (dense-equivalent bytes)", 32, O.OPT_MASKED, prob, pf.RKL2, "rkl2", 5),
            ("rkl2 mobility-weighted projection FP32 (generic)", 32, 0, prob.with_(simplex=1), pf.RKL2, "rkl2", 5),
            ("rkl2 FP64 (generic)", 64, 0, prob, pf.RKL2, "rkl2", 5),
            ("ssp(10)4 stage FP32 (one-cell rolled, with z)", 32, 0, prob, pf.SSP104, "ssp", 4),
            ("ssp(10)4 stage FP32 masked", 32, O.OPT_MASKED, prob, pf.SSP104, "ssp", 4)]
    out = {"workload": prob.name, "peak_gbs": peak, "passes": []}
    for name, prec, opts, p, integ, kind, nvec in runs:
        sim = pf.Simulation(p, precision=prec, stream=stream, options=opts)
        sim.set_state(u)
        sim.step(integ, 1e30, tol=TOL, max_attempts=1)
        torch.cuda.synchronize()
        sim.profile(1)
        for _ in range(2):
            sim.step(integ, 1e30, tol=TOL, max_attempts=1)
        prof = sim.profile(0)
        sim.close()
        ms, n = prof.get(kind, (0.0, 0))
        if not n:
            continue
        nbytes = nvec * N * (prec // 8) * V
        ach = nbytes / (ms / n * 1e-3) / 1e9
        row = {"pass": name, "ms": ms / n, "launches": n, "bytes": nbytes}
        if opts & O.OPT_MASKED:
            # masked storage moves fewer bytes than the dense ones counted here:
            # a rate, not a fraction of the memory bandwidth
            row["dense_equivalent_gbs"] = ach
        else:
            row.update({"gbs": ach, "frac_of_measured_peak": ach / peak})
        out["passes"].append(row)
    # the energy functional (Eq. energy): one FP32 state read per evaluation
    sim = pf.Simulation(prob, precision=32, stream=stream)
    sim.set_state(u)
    sim.energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        sim.energy()
    el = (time.perf_counter() - t0) / 3
    sim.close()
    nbytes = N * 4 * V
    out["passes"].append({"pass": "energy functional FP32 (one call, host round trip included)", "ms": 1e3 * el,
                          "bytes": nbytes, "gbs": nbytes / el / 1e9, "frac_of_measured_peak": nbytes / el / 1e9 / peak})
    return out


def _peak_gbs():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
    except (OSError, ValueError):
        return 6800.0


def masked_run(pf, torch, prob, u, stream, args, world, dev, dense_out, dense_pass_ms):
    """The bench steps again in masked storage (PF_OPT_MASKED) from the same
    initial state: GCell-updates/s, per-pass times, and the largest
    difference from the dense run's final state (the masked kernels share the
    one-cell kernels' arithmetic, the dense run takes the two-cell kernels:
    FP32 rounding differences, which the discontinuous activity filter can
    turn into O(1e-3) local ones)."""
    V, N = prob.V, prob.n_phases
    sim = pf.Simulation(prob, precision=32, stream=stream, options=pf.Simulation.OPT_MASKED)
    sim.set_state(u)
    for _ in range(args.warmup):
        sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1)
    torch.cuda.synchronize()
    barrier(world)
    sim.profile(1)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sweeps = 0
    for _ in range(args.steps):
        sweeps += sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1)["rhs_evals"]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    prof = sim.profile(0)
    out = torch.empty_like(dense_out)
    sim.get_state(out=out)
    torch.cuda.synchronize()         # the copy runs on the simulation's stream
    d = (out - dense_out).abs()
    diff = {"max": float(d.max()), "mean": float(d.mean())}
    del d
    sim.close()
    occ = float((u[:N] != 0).sum(0, dtype=torch.float64).mean())
    pass_ms = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1] > 0}
    rk = pass_ms.get("rkl2")
    dk = dense_pass_ms.get("rkl2")
    return {"value": aggregate_value(V, sweeps, ms, world), "unit": UNIT, "ms_per_step": ms / args.steps,
            "sweeps": sweeps, "pass_ms": pass_ms, "abs_diff_to_dense": diff,
            "rkl2_pass_speedup": (dk["ms"] / dk["launches"]) / (rk["ms"] / rk["launches"]) if rk and dk else None,
            "mean_nonzero_phases_per_cell": occ,
            "storage": "dense phase planes + one 32-bit occupancy word per cell and vector"}


def reuse_run(pf, torch, prob, u, stream, args, world, dev, dense_out, dense_ms):
    """The bench steps again with F(u^{n+1}) of each accepted step reused as
    the next step's F(u^n) (PF_STEP_REUSE_RHS): time per step, RHS sweeps,
    and the largest difference from the dense run's final state."""
    V = prob.V
    sim = pf.Simulation(prob, precision=32, stream=stream)
    sim.set_state(u)
    f = pf.Simulation.STEP_REUSE_RHS
    for _ in range(args.warmup):
        sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1, flags=f)
    torch.cuda.synchronize()
    barrier(world)
    sim.profile(1)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sweeps, stages, accepted = 0, [], 0
    for _ in range(args.steps):
        st = sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1, flags=f)
        sweeps += st["rhs_evals"]
        stages.append(st["rhs_evals"])
        accepted += st["steps_accepted"]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    prof = sim.profile(0)
    out = torch.empty_like(dense_out)
    sim.get_state(out=out)
    torch.cuda.synchronize()         # the copy runs on the simulation's stream
    d = (out - dense_out).abs()
    mean_diff = float(d.mean())
    frac = float((d.amax(0) > 1e-3).double().mean())
    del d
    sim.close()
    # the RHS is discontinuous (activity filter, clamps), so rounding-level
    # differences flip a few cells; the bulk of the state agrees to rounding
    return {"ms_per_step": ms / args.steps, "dense_ms_per_step": dense_ms / args.steps, "rhs_sweeps": sweeps,
            "sweeps_per_step": stages, "accepted": accepted,
            "value": aggregate_value(V, sweeps, ms, world), "unit": UNIT,
            "pass_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1] > 0},
            "mean_abs_diff_to_dense": mean_diff, "cells_differing_over_1e-3": frac}


def stefan_sweep(pf, torch, t_end=43e3, full=False):
    """The Stefan strip (1024 x 256, D 1:100) to the configuration's t_end
    (43e3, front advance X ~ 50) with ten output times: forward Euler at
    0.9 dt_e in FP64 and FP32, SSP(5)2 at 3.6 dt_e, and the adaptive schemes
    at r = a in {1e-3 .. 1e-6}: wall time, RHS sweeps, steps, the error of the
    fitted growth constant against the exact A, and the speed-up over FP64
    forward Euler of every run whose error is within 1.05x of its error.
    The default list is a bounded subset (RKL2 FP32 at every tolerance, RKL2
    FP64, RKL1 and SSP(10)4 FP32 at 1e-3); full=True runs every integrator at
    every tolerance in both precisions."""
    import numpy as np
    from paper_2601_16522_gb300 import inputs as I
    prob, u = I.stefan(1024, 256, 200.0)
    A = I.stefan_growth_constant()
    x0 = _front(u[0][:1024])
    stream = torch.cuda.Stream()
    times = np.linspace(0.0, t_end, 11)[1:]
    runs = [("feuler", 64, None, dict(dt_mult=0.9)), ("feuler", 32, None, dict(dt_mult=0.9)),
            ("ssp2", 32, None, dict(dt_mult=3.6, ssp_stages=5))]
    if full:
        for tol in (1e-3, 1e-4, 1e-5, 1e-6):
            for integ in ("rkl1", "rkl2", "ssp104"):
                for prec in (32, 64):
                    runs.append((integ, prec, tol, dict(tol=(tol, tol, tol, tol))))
    else:
        for tol in (1e-3, 1e-4, 1e-5, 1e-6):
            runs.append(("rkl2", 32, tol, dict(tol=(tol, tol, tol, tol))))
        for integ, prec in (("rkl2", 64), ("rkl1", 32), ("ssp104", 32)):
            runs.append((integ, prec, 1e-3, dict(tol=(1e-3,) * 4)))
    out = []
    host = np.zeros((3, prob.V))
    for name, prec, tol, kw in runs:
        integ = {"feuler": pf.FEULER, "ssp2": pf.SSP2, "rkl1": pf.RKL1, "rkl2": pf.RKL2, "ssp104": pf.SSP104}[name]
        sim = pf.Simulation(prob, precision=prec, stream=stream)
        sim.set_state(u)
        X, evals, acc, rej = [], 0, 0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for tk in times:
            st = sim.step(integ, float(tk), **kw)
            evals += st["rhs_evals"]
            acc += st["steps_accepted"]
            rej += st["steps_rejected"]
            sim.get_state(out=host)
            X.append(_front(host[0][:1024]) - x0)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        sim.close()
        Afit = float((np.sqrt(times) * np.array(X)).sum() / times.sum())
        out.append({"integrator": name, "precision": prec, "tol": tol, "wall_ms": 1e3 * el, "rhs_evals": evals,
                    "accepted": acc, "rejected": rej, "rel_error": abs(Afit - A) / A})
    ref = out[0]
    for r in out:
        r["speedup_vs_fe64"] = ref["wall_ms"] / r["wall_ms"]
        r["at_target_error"] = bool(r["rel_error"] <= 1.05 * ref["rel_error"] + 1e-12)
    ok = [r for r in out if r["at_target_error"]]
    best = min(ok, key=lambda r: r["wall_ms"])
    return {"t_end": t_end, "A_exact": A, "target_error": ref["rel_error"], "runs": out,
            "fastest_at_target": {k: best[k] for k in ("integrator", "precision", "tol", "speedup_vs_fe64")}}


def grains_to_half(pf, torch, dev, stream, t_max=60.0, wall_cap_s=120.0, full=False):
    """The 256^3 grain workload run to the time at which half of the 32
    grains are gone (alive: max phi_a >= 0.5; the configuration's run
    length), adaptive RKL2 in FP32 with masked and with dense storage,
    adaptive RKL1 and SSP(10)4 in masked storage (each stops at the wall cap);
    forward Euler in FP64 at 0.9 dt_e is estimated from its measured time
    per step times the steps it would need."""
    prob, u, _ = workload_problem("grains256", dev)
    out = []
    t_half = None
    runs = [("rkl2-fp32-masked", pf.RKL2, pf.Simulation.OPT_MASKED)]
    if full:
        runs.append(("rkl2-fp32-dense", pf.RKL2, 0))
    runs.append(("rkl1-fp32-masked", pf.RKL1, pf.Simulation.OPT_MASKED))
    runs.append(("ssp104-fp32-masked", pf.SSP104, pf.Simulation.OPT_MASKED))
    for name, integ, opts in runs:
        sim = pf.Simulation(prob, precision=32, stream=stream, options=opts)
        sim.set_state(u)
        dte = sim.dt_e()
        n0 = sim.reduce()[2]
        dt_out = 200.0 * dte
        t, evals, alive = 0.0, 0, n0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cap = wall_cap_s if integ != pf.SSP104 or full else 0.5 * wall_cap_s
        while alive > n0 // 2 and t < t_max and time.perf_counter() - t0 < cap:
            t += dt_out
            evals += sim.step(integ, t, tol=TOL)["rhs_evals"]
            alive = sim.reduce()[2]
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        sim.close()
        out.append({"variant": name, "wall_s": el, "t_reached": t, "grains_alive": alive, "grains_start": n0,
                    "rhs_evals": evals})
        if integ == pf.RKL2:
            t_half = t if alive <= n0 // 2 else t_half
    # fixed-step schemes, FP32 masked: 20 timed steps each at their largest
    # stable step (SSP(5)2 at 4 dt_e, Sec. 3.2), extrapolated to t_half
    for name, integ, mult in (("feuler-fp32-masked (estimated)", pf.FEULER, 0.9),
                              ("ssp52-fp32-masked (estimated)", pf.SSP2, 3.6)):
        sim = pf.Simulation(prob, precision=32, stream=stream, options=pf.Simulation.OPT_MASKED)
        sim.set_state(u)
        dte = sim.dt_e()
        sim.step(integ, 2 * mult * dte, dt_mult=mult)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sim.step(integ, 22 * mult * dte, dt_mult=mult)
        torch.cuda.synchronize()
        per_step = (time.perf_counter() - t0) / 20.0
        sim.close()
        if t_half is not None:
            n = math.ceil(t_half / (mult * dte))
            out.append({"variant": name, "wall_s": per_step * n, "rhs_evals": n * st["rhs_evals"] // 20,
                        "ms_per_step": 1e3 * per_step, "dt": "%g dt_e" % mult})
    # forward Euler, FP64, dense: 20 timed steps, extrapolated
    sim = pf.Simulation(prob, precision=64, stream=stream)
    sim.set_state(u)
    dte = sim.dt_e()
    sim.step(pf.FEULER, 2 * 0.9 * dte, dt_mult=0.9)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(pf.FEULER, 22 * 0.9 * dte, dt_mult=0.9)
    torch.cuda.synchronize()
    per_step = (time.perf_counter() - t0) / 20.0
    sim.close()
    if t_half is not None:
        n_fe = math.ceil(t_half / (0.9 * dte))
        out.append({"variant": "feuler-fp64-dense (estimated)", "wall_s": per_step * n_fe, "rhs_evals": n_fe,
                    "ms_per_step": 1e3 * per_step})
    return {"t_half": t_half, "output_interval": "200 dt_e", "tol": TOL, "variants": out}


def sinter_horizon(pf, torch, dev, stream, t_r=0.05, wall_cap_s=150.0):
    """The 320^3 sintering workload (64 grains + one pore phase + c) run
    with adaptive RKL2 in FP32 masked storage at r = a = 1e-4 towards the
    horizon t_r (the configuration's t_r = 0.05 is about 1.8e5 stable Euler
    steps), in output intervals of 0.0025, until the wall-clock cap; the time
    reached, RHS sweeps against forward Euler's and the conserved totals are
    reported."""
    prob, u, _ = workload_problem("sinter320", dev)
    N = prob.n_phases
    tol = (1e-4, 1e-4, 1e-4, 1e-4)
    sim = pf.Simulation(prob, precision=32, stream=stream, options=pf.Simulation.OPT_MASKED)
    sim.set_state(u)
    dte = sim.dt_e()
    m0, vol0, alive0 = sim.reduce()
    t, evals, acc, rej, status = 0.0, 0, 0, 0, "reached t_r"
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while t < t_r:
        if time.perf_counter() - t0 > wall_cap_s:
            status = "wall-clock cap"
            break
        try:
            st = sim.step(pf.RKL2, min(t_r, t + 0.0025), tol=tol)
        except pf.PfError as e:
            status = "stopped: %s" % e
            break
        evals += st["rhs_evals"]
        acc += st["steps_accepted"]
        rej += st["steps_rejected"]
        t = st["t"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    m1, vol1, alive1 = sim.reduce()
    sim.close()
    return {"workload": prob.name, "cells": prob.V, "phases": N, "pores": prob.pores, "porosity": prob.porosity,
            "dt_e": dte, "tol": tol, "t_r": t_r, "t_reached": t, "status": status, "rhs_evals": evals,
            "accepted": acc, "rejected": rej, "wall_s": wall, "fe_rhs_evals": t / dte,
            "rhs_ratio_vs_fe": (t / dte) / max(evals, 1), "gcell_updates_per_s": prob.V * evals / wall / 1e9,
            "grains_alive": [alive0, alive1],
            "pore_volume_change": float((vol1[N - 1] - vol0[N - 1]) / vol0[N - 1]),
            "solute_change": float(abs(m1 - m0) / m0)}


def zener_sts(pf, torch, dev, stream, n=128, n_grains=32, t_eq=0.5, t_run=10.0, full=False):
    """Grain growth with immobile particles (Sec. 5.3, Zener pinning; the
    paper's 11.5x case, Tab. perf-ggpores, on a 400^3 domain to t_r = 884):
    n^3 cells, particles of radius 6 at volume fraction 0.15, masked FP32
    storage.  The equilibration run of Sec. 5.3 (its parameters, adaptive
    RKL2 to t_eq; the paper's 5 time units with full=True) is followed by
    the immobile run with adaptive RKL2 over t_run time units; the RHS sweeps
    are compared with the stable Euler steps the same interval takes
    (t_run / dt_e).  More than 12 nontrivial phases per cell appear at the
    particle fringes under the STS schemes; those cells take the wide path.
    With full=True the first time unit of the immobile run is repeated with
    the mobility-weighted projection (dense storage, generic passes) beside
    the standard one."""
    if full:
        t_eq = 5.0
    from paper_2601_16522_gb300 import inputs as I
    prob, u = I.zener_device(n=n, n_grains=n_grains, device=dev)
    opts = pf.Simulation.OPT_MASKED
    eq = pf.Simulation(I.zener_equilibration(prob), precision=32, stream=stream, options=opts)
    eq.set_state(u)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_eq = eq.step(pf.RKL2, t_eq, tol=(1e-4, 1e-2, 1e-4, 1e-3))
    u1 = torch.empty_like(u)
    eq.get_state(out=u1)
    torch.cuda.synchronize()
    eq.close()
    sim = pf.Simulation(prob, precision=32, stream=stream, options=opts)
    dte = sim.dt_e()
    sim.set_state(u1, t=0.0)
    evals, acc, rej = 0, 0, 0
    tol = (1e-4, 1e-2, 1e-4, 1e-3)
    t1 = time.perf_counter()
    for k in range(1, 11):
        st = sim.step(pf.RKL2, k * t_run / 10, tol=tol)    # ten output times
        evals += st["rhs_evals"]
        acc += st["steps_accepted"]
        rej += st["steps_rejected"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t1
    _, _, nz = sim.get_state(out=torch.empty_like(u1), with_nz=True)
    torch.cuda.synchronize()
    sim.close()
    # the first time unit with each projection (dense storage, same state)
    proj = {}
    for name, p in ((("standard", prob), ("mobility-weighted", prob.with_(simplex=1))) if full else ()):
        sim = pf.Simulation(p, precision=32, stream=stream)
        sim.set_state(u1, t=0.0)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        st = sim.step(pf.RKL2, 1.0, tol=tol)
        torch.cuda.synchronize()
        _, _, nzp = sim.get_state(out=torch.empty_like(u1), with_nz=True)
        torch.cuda.synchronize()
        proj[name] = {"t": 1.0, "rhs_evals": st["rhs_evals"], "accepted": st["steps_accepted"],
                      "rejected": st["steps_rejected"], "wall_s": time.perf_counter() - t2,
                      "max_nontrivial_phases_per_cell": int(nzp.max().item())}
        sim.close()
    fe = t_run / dte
    return {"workload": prob.name, "cells": prob.V, "phases": prob.n_phases, "dt_e": dte, "tol": tol,
            "equilibration": {"t": t_eq, "rhs_evals": st_eq["rhs_evals"], "wall_s": t1 - t0},
            "t_run": t_run, "rhs_evals": evals, "accepted": acc, "rejected": rej, "wall_s": wall,
            "fe_steps": fe, "rhs_ratio_vs_fe": fe / max(evals, 1), "paper_ratio": 14110453 / 1224604,
            "max_nontrivial_phases_per_cell": int(nz.max().item()), "projections": proj}


def slots_many_grains(pf, torch, dev, stream, n=256, n_grains=2000, attempts=6):
    """Slot storage (Sec. 3.1: 12 phase values and ids per cell) on a grain
    structure with many more grains than dense planes could hold: n^3 cells,
    n_grains Voronoi grains, adaptive RKL2 in FP32.  Reports the device
    footprint beside that of dense storage, GCell-updates/s over a few
    attempts after one warm-up attempt, and the RKL2 pass's algorithmic
    bandwidth (5 slot vectors of 72 B per cell)."""
    from paper_2601_16522_gb300 import inputs as I
    t0 = time.perf_counter()
    prob, vals, ids, _ = I.grains_slots_device(n=n, n_grains=n_grains, seed=7, device=dev)
    build_s = time.perf_counter() - t0
    opts = pf.Simulation.OPT_SLOTS
    fp = pf.footprint(prob, 32, options=opts)
    dense = 5 * prob.V * n_grains * 4
    sim = pf.Simulation(prob, precision=32, stream=stream)
    sim.set_state_slots(vals, ids)
    del vals, ids
    _, _, alive0 = sim.reduce()
    sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1)
    torch.cuda.synchronize()
    sim.profile(1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sweeps = 0
    for _ in range(attempts):
        sweeps += sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1)["rhs_evals"]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = sim.profile(0)
    _, _, alive = sim.reduce()
    sim.close()
    out = {"workload": prob.name, "cells": prob.V, "grains": n_grains, "slots_per_cell": 12,
           "footprint_gb": fp / 1e9, "dense_state_vectors_gb": dense / 1e9, "build_s": build_s,
           "attempts": attempts, "rhs_evals": sweeps, "ms": ms,
           "gcell_updates_per_s": prob.V * sweeps / (ms * 1e-3) / 1e9, "grains_alive": [alive0, alive]}
    if prof.get("rkl2", (0, 0))[1]:
        per = prof["rkl2"][0] / prof["rkl2"][1]
        out["rkl2_pass_ms"] = per
        out["rkl2_pass_gbs"] = 5 * 72 * prob.V / (per * 1e-3) / 1e9
    return out


def precision_check(pf, torch, dev, stream, t_end=2.0):
    """FP32 against FP64 on the 256^3 grain workload: adaptive RKL2 from the
    same initial state to the same time t_end (about 2400 stable Euler steps)
    in FP32 (masked storage, equal to dense) and in FP64; the largest
    difference of any phase value, the largest relative difference of a
    phase volume and the alive-grain counts."""
    prob, u, _ = workload_problem("grains256", dev)
    out = {}
    res = {}
    for prec, opts in ((32, pf.Simulation.OPT_MASKED), (64, 0)):
        sim = pf.Simulation(prob, precision=prec, stream=stream, options=opts)
        sim.set_state(u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sim.step(pf.RKL2, t_end, tol=TOL)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        _, vol, alive = sim.reduce()
        v = torch.empty_like(u)
        sim.get_state(out=v)
        torch.cuda.synchronize()
        sim.close()
        res[prec] = (v, vol, alive)
        out["fp%d" % prec] = {"rhs_evals": st["rhs_evals"], "accepted": st["steps_accepted"],
                              "rejected": st["steps_rejected"], "wall_s": wall, "grains_alive": alive}
    d = (res[32][0] - res[64][0]).abs()
    vol32, vol64 = res[32][1], res[64][1]
    out.update({"t_end": t_end, "max_abs_phi_diff": float(d.max().item()),
                "mean_abs_phi_diff": float(d.mean().item()),
                "max_rel_volume_diff": float(max(abs(a - b) / b for a, b in zip(vol32, vol64) if b > 0))})
    return out


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2601_16522_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2601_16522_gb300 import pf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prob, u, prec = workload_problem(args.workload, dev)
    V, N = prob.V, prob.n_phases
    sim = pf.Simulation(prob, precision=prec, stream=stream,
                        options=pf.Simulation.OPT_TMA if args.tma else 0)
    torch.cuda.synchronize()
    sim.set_state(u)
    torch.cuda.synchronize()
    tuned = None
    if not args.tma and not args.no_autotune:
        choice, ms = sim.autotune()
        names = ["two_cell", "one_cell", "tma"]
        tuned = {"choice": names[choice]}
        tuned.update({"rkl2_pass_ms_" + names[k]: v for k, v in ms.items()})

    def one_step():
        return sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    barrier(world)

    clocks = ClockSampler(local)
    clocks.start()
    sim.profile(1)
    l0 = sim.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(stream)
    sweeps, ss, acc = 0, [], 0
    for _ in range(args.steps):
        st = one_step()
        sweeps += st["rhs_evals"]
        acc += st["steps_accepted"]
        ss.append(st["rhs_evals"])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    launches = sim.launch_count() - l0
    prof = sim.profile(0)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, world, dev)
    value = aggregate_value(V, sweeps, ms_max, world)

    # roofline of the dominant pass kind
    kinds = {k: v for k, v in prof.items() if v[1] > 0 and k in PASS_VECTORS}
    dom = max(kinds, key=lambda k: kinds[k][0]) if kinds else None
    vec_bytes = V * (N + prob.has_conc) * (4 if prec == 32 else 8)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = None
    if dom:
        ms_k, n_k = kinds[dom]
        bytes_launch = PASS_VECTORS[dom] * vec_bytes
        achieved = bytes_launch / (ms_k / n_k * 1e-3) / 1e9
        variant = "tma" if args.tma else (tuned["choice"] if tuned else "two_cell")
        traffic = None
        if dom == "rkl2" and args.workload in RKL2_TRAFFIC_PER_CELL and variant == "two_cell":
            traffic = RKL2_TRAFFIC_PER_CELL[args.workload] * V
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kernel_name(prob, prec, variant) + " (%s pass)" % dom,
                "bytes_per_launch": bytes_launch, "avg_launch_ms": ms_k / n_k,
                "frac_of_spec_8tbs": achieved / 8000.0,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    pass_ms = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1] > 0}

    # masked storage (the GPU form of the per-cell phase lists): the same
    # steps from the same state; its result must equal the dense one
    masked = None
    reuse = None
    if not args.no_masked and prec == 32 and N <= 128:
        dense_out = torch.empty((N + prob.has_conc, V), dtype=torch.float64, device=dev)
        sim.get_state(out=dense_out)
        torch.cuda.synchronize()
        masked = masked_run(pf, torch, prob, u, stream, args, world, dev, dense_out, pass_ms)
        if not args.no_reuse:
            reuse = reuse_run(pf, torch, prob, u, stream, args, world, dev, dense_out, ms_max)
        del dense_out

    # end-to-end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_in = torch.empty((N + prob.has_conc, V), dtype=torch.float64, pin_memory=True)
        host_out = torch.empty_like(host_in, pin_memory=True)
        host_in.copy_(u.to("cpu"))
        # settled step size: the controller's current proposal
        st_probe = sim.step(pf.RKL2, 1e30, tol=TOL, max_attempts=1)
        dt_settled = st_probe["dt_next"]
        torch.cuda.synchronize()
        n_e2e = max(1, min(args.steps, 3))
        e_sweeps = 0
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            sim.set_state(host_in, 0.0)
            st = sim.step(pf.RKL2, 1e30, tol=TOL, dt0=dt_settled, max_attempts=1)
            e_sweeps += st["rhs_evals"]
            sim.get_state(out=host_out.numpy())
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world, dev)
        bi = host_in.numel() * 8
        e2e = {"value": world * V * e_sweeps / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bi, "steps": n_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on all host cores (OpenMP over the RHS rows) and on one
        m = 64 if N <= 32 else 32
        sub, us = sub_box(prob, u, m)
        from oracle import ref
        ref.set_openmp(True)
        try:
            v, el, sw = oracle_sample(us, sub)
        finally:
            ref.set_openmp(False)
        ms1 = 48 if N <= 32 else 24
        sub1, us1 = sub_box(prob, u, ms1)
        v1, el1, _ = oracle_sample(us1, sub1)
        cores = os.cpu_count()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one RKL2 step (s=5) + error sweep on a %d^3 sub-box of the same state, %.1f s, "
                         "OpenMP on all %d host cores (RHS rows shared)" % (m, el, cores),
               "single_thread": {"value": v1, "cores": 1,
                                 "sample": "the same step on a %d^3 sub-box, %.1f s" % (ms1, el1)}}

    extras = rank == 0 and world == 1 and not args.quick
    tts = None
    if extras and not args.no_tts:
        tts = time_to_solution(pf, torch)
    served = None
    if extras and args.served > 0:
        served = served_stream(pf, torch, args.served)
    to_half = None
    if extras and not args.no_grains_to_half:
        to_half = grains_to_half(pf, torch, dev, stream, full=args.full)
    sweep = None
    if extras and not args.no_stefan_sweep:
        sweep = stefan_sweep(pf, torch, full=args.full)
    horizon = None
    if extras and not args.no_sinter:
        horizon = sinter_horizon(pf, torch, dev, stream, t_r=0.05 if args.full else 0.01)
    prec_check = None
    if extras and args.precision_check:
        prec_check = precision_check(pf, torch, dev, stream)
    fe64 = None
    if extras:
        fe64 = fp64_fe_pass(pf, torch, dev, stream)
    zener = None
    if extras and not args.no_zener:
        zener = zener_sts(pf, torch, dev, stream, full=args.full)
    slots = None
    if extras and not args.no_slots:
        slots = slots_many_grains(pf, torch, dev, stream)
    oracle_cfg = None
    if extras and not args.no_cpu_baseline:
        oracle_cfg = oracle_configs()
    families = None
    if extras:
        families = kernel_families(pf, torch, dev, stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == 32 else "f64",
            "data": "synthetic",
            "config": {"workload": "3D %s %s: %dx%dx%d periodic, %d dense phases%s, FP32 storage, "
                                   "adaptive RKL2 (tol r=%g a_phi=%g)" % (
                                       "sintering (grains + pores + vacancy concentration)"
                                       if args.workload.startswith("sinter") else "grain growth",
                                       args.workload, prob.nx, prob.ny, prob.nz, N,
                                       " + 1 concentration" if prob.has_conc else "", TOL[0], TOL[1]),
                       "cells": V, "phases": N, "integrator": "rkl2-adaptive", "parallelism": "replicas",
                       "l2": "state vectors %.2f GB each > L2 (no flush needed)" % (vec_bytes / 1e9),
                       "autotune": tuned},
            "sweeps": sweeps, "stages_per_step": ss, "accepted": acc,
            "roofline": roof, "pass_ms": pass_ms,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "time_to_solution": tts, "served": served, "masked": masked, "reuse_rhs": reuse,
            "grains_to_half": to_half, "stefan_sweep": sweep, "sinter_horizon": horizon, "precision_check": prec_check,
            "fp64_fe_pass": fe64, "zener_sts": zener, "slots_many_grains": slots, "oracle_configs": oracle_cfg,
            "kernel_families": families,
        }
        print(json.dumps(line), flush=True)
    sim.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grains256")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tma", action="store_true", help="TMA-staged kernels instead of plain loads")
    ap.add_argument("--no-tts", action="store_true", help="skip the 2D time-to-solution runs")
    ap.add_argument("--served", type=int, default=2000, help="requests in the served Poisson stream (0: skip)")
    ap.add_argument("--quick", action="store_true", help="only the headline steps (no configuration runs)")
    ap.add_argument("--full", action="store_true",
                    help="full configuration runs: every integrator/tolerance of the Stefan sweep, dense RKL2 "
                         "to t_half, sintering to t_r = 0.05")
    ap.add_argument("--no-grains-to-half", action="store_true")
    ap.add_argument("--no-stefan-sweep", action="store_true")
    ap.add_argument("--no-sinter", action="store_true")
    ap.add_argument("--no-zener", action="store_true")
    ap.add_argument("--no-slots", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel variant (two cells per thread) instead of timing the variants "
                         "first (a profiler distorts those timings)")
    ap.add_argument("--no-masked", action="store_true", help="skip the masked-storage run")
    ap.add_argument("--no-reuse", action="store_true", help="skip the run that reuses F(u^{n+1})")
    ap.add_argument("--precision-check", action="store_true",
                    help="256^3 grain workload: FP32 against FP64, adaptive RKL2 to t = 2")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
