"""Benchmark of the FB-LTS hot path on GB300: cell-updates/s, % of HBM peak, latency.

One step = one coarse FB-LTS step (coarse advancement, interface prediction,
M fine subcycles with the correction sums, interface correction) of the whole
synthetic workload, through the C ABI.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fblts|reference]
                  [--workload shelf|bump] [--precision fp64|fp32]

With N > 1 (torchrun) every rank advances its own replica of the workload
(the method has no cross-replica exchange); value = all ranks' cell-updates
divided by the slowest rank's time.  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SWE cell-updates/s (% HBM peak), FP32 vs FP64 at stated err; p50/p99 latency"
UNIT = "cell-updates/s"


def make_workload(name, build=True):
    """The named synthetic workload and its description (build=False: the
    description only)."""
    from synth import basin, scenario
    table = {
        "shelf": (scenario.shelf_case,
                  "periodic-in-y 512x512 hex channel, dc 2 km, walls in x, tanh shelf 10-4000 m with 5% "
                  "roughness, 2 LTS levels (M=4) by gravity-wave CFL, 15 m/s wind stress + quadratic drag"),
        "basin": (basin.basin_case,
                  "closed basin, variable-resolution Voronoi mesh (~2.0M cells): 500 m along a seeded sinuous "
                  "coast growing to 20 km offshore, depth 5-4000 m, 3 LTS levels (M=8) by gravity-wave CFL, "
                  "moving Holland vortex with wind stress, pressure gradient and quadratic drag"),
        "basin_half": (lambda: basin.basin_case(Ly=4800e3),
                       "1/2-length sample of the basin workload (same recipe, Ly 4800 km, ~1.0M cells)"),
        "basin_small": (lambda: basin.basin_case(Ly=1200e3),
                        "1/8-length sample of the basin workload (same recipe, Ly 1200 km, ~0.25M cells)"),
        "basin_tiny": (lambda: basin.basin_case(Ly=150e3),
                       "1/64-length sample of the basin workload (same recipe, Ly 150 km, ~32k cells)"),
        "bump": (lambda: scenario.gaussian_bump_case(two_level=True),
                 "doubly periodic 32x32 hex, flat 1000 m, Gaussian bump, 2 LTS levels (M=2)"),
    }
    if name not in table:
        raise SystemExit(f"unknown workload {name}")
    make, desc = table[name]
    return (make() if build else None), desc


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# sources of the single-state kernels (their bodies, launches and tables)
KERNEL_SOURCES = ("fblts_internal.h", "kernels.cuh", "kernel_bodies.cuh", "kernel_bodies32.cuh", "kernels.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2405_10505_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(workload, precision, kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if current."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(f"{workload}/{precision}/{kernel}")
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def oracle_sample(s, budget_s=15.0, threads=1):
    """Times the FP64 oracle on whole coarse steps of the workload.

    The oracle is single-threaded; with threads > 1 one instance per thread
    advances its own copy of the state (the C library runs without the
    interpreter lock), so the host's cores all work, as replicas.  The step
    count comes from a one-step probe (none when budget_s <= 0: one step);
    the timed run then takes all its steps in one oracle call, so the state
    stays in the oracle's own representation throughout.  Returns the steps
    of all instances, the wall time of the timed runs, and the state and step
    count of the first instance."""
    import threading

    import oracle
    m = oracle.Mesh.from_scenario(s)
    p = oracle.scenario_params(s)
    oracle.lib()
    n = 1
    if budget_s > 0:
        tp = time.perf_counter()
        oracle.fblts(m, p, s.level, s.M, s.h0, s.u0, s.dt, 1)
        n = int(max(1, min(50, budget_s / max(time.perf_counter() - tp, 1e-9))))
    out = [None] * threads
    t0 = time.perf_counter()

    def run(i):
        try:
            h, u = oracle.fblts(m, p, s.level, s.M, s.h0, s.u0, s.dt, n)
            out[i] = (n, h, u)
        except BaseException as exc:      # re-raised below, in the calling thread
            out[i] = exc

    workers = [threading.Thread(target=run, args=(i,)) for i in range(threads)]
    for w in workers:
        w.start()
    for w in workers:
        w.join()
    el = time.perf_counter() - t0
    for o in out:
        if isinstance(o, BaseException):
            raise o
    return sum(o[0] for o in out), el, out[0][1], out[0][2], out[0][0]


def cpu_threads(args):
    """Oracle instances for the CPU legs: --cpu-threads, else one per host core."""
    return args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)


def forcing_flags(s):
    import paper_2405_10505_gb300 as fb
    fz = s.forcing
    return ((fb.FORCE_WIND_STRESS if fz.wind_stress else 0) | (fb.FORCE_BOTTOM_DRAG if fz.cd else 0)
            | (fb.FORCE_VORTEX if fz.vortex is not None else 0))


def cell_updates_per_step(s):
    counts = np.bincount(s.level, minlength=s.nLevels)
    mult, cu = 1, 0
    for l in range(s.nLevels):
        cu += int(counts[l]) * mult
        if l + 1 < s.nLevels:
            mult *= s.M[l]
    return cu


# classical RK4 is stable on the imaginary axis up to |omega dt| = 2 sqrt(2)
RK4_IMAG_LIMIT = 2.0 * np.sqrt(2.0)


def fbrk32_imag_limit(beta):
    """Largest omega*dt for which one FB-RK(3,2) step (Eq. fbrk32, FB weights
    beta) of the oscillator h' = u, u' = -h does not amplify: the linear
    gravity-wave limit, used to put RK4 at the same fraction of its own limit."""
    b1, b2, b3 = beta

    def step(h, u, t):
        h1 = h + t / 3 * u
        u1 = u - t / 3 * (b1 * h1 + (1 - b1) * h)
        h2 = h + t / 2 * u1
        u2 = u - t / 2 * (b2 * h2 + (1 - b2) * h)
        h3 = h + t * u2
        u3 = u - t * (b3 * h3 + (1 - 2 * b3) * h2 + b3 * h)
        return h3, u3

    def rho(t):
        return max(abs(np.linalg.eigvals(np.array([step(1.0, 0.0, t), step(0.0, 1.0, t)]).T)))

    lo, hi = 0.5, 6.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if rho(mid) <= 1 + 1e-12 else (lo, mid)
    return lo


def reference_sample(workload):
    """The workload the oracle times per step: the workload itself, or for the
    2M-cell basin (about 100 s per oracle coarse step) its 1/64-length sample
    (about 1.5 s per step, so a run of ~100 steps ends within a few minutes)."""
    if workload == "basin":
        ws, _ = make_workload("basin_tiny")
        return ws, "basin_tiny (1/64-length sample of the basin: same recipe, Ly 150 km, 31.7k cells)"
    ws, _ = make_workload(workload)
    return ws, workload


def run_reference(args, rank):
    """The reference arm: the oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    _, desc = make_workload(args.workload, build=False)
    ws, sample_name = reference_sample(args.workload)
    T = cpu_threads(args)
    for _ in range(args.warmup):
        oracle_sample(ws, budget_s=0.0, threads=T)
    cu = cell_updates_per_step(ws)
    steps, walls = [], []
    for k in range(args.steps):
        n, el, _, _, _ = oracle_sample(ws, budget_s=0.0, threads=T)
        steps.append(n)
        walls.append(el)
    ms = 1000.0 * statistics.mean(walls)     # one timed step: a coarse step on every instance
    v = cu * sum(steps) / sum(walls)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": T, "kind": "oracle",
                             "sample": f"{args.steps} steps, each one whole coarse step of {sample_name} on each "
                                       f"of {T} threads (one single-threaded C oracle instance per host core)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def max_over_ranks(ms, dist, torch, device):
    """The slowest rank's time: every rank contributes its own and gets the max."""
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, cell_updates_per_step, steps, ms_total):
    """Whole-job throughput of `world` independent replicas, timed by the slowest."""
    return world * cell_updates_per_step * steps / (ms_total / 1000.0)


def timed_steps(fb, torch, st, stream, warm, k):
    """Mean device time (ms) of one step over k steps after `warm` untimed ones."""
    fb.lts_advance(st, warm)
    fb.synchronize(st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fb.lts_advance(st, k)
    e1.record(stream)
    fb.synchronize(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def run_ensemble(args, rank):
    """Batched ensemble: `--members` shelf channels of seeded sizes (20k-800k
    cells), vortex tracks and M in {2, 4, 8}, FP32-tendency.  Times rounds of
    one coarse step of every member in three forms, all with CUDA events:
    plain concurrent (each member's captured step on its own stream, joined
    per round), plain sequential (every member's captured step on one stream,
    one instance per launch after another), and the batch (fblts_batch_*,
    launch shape tuned online)."""
    if rank != 0:
        return
    import torch
    import paper_2405_10505_gb300 as fb
    from synth import scenario
    torch.cuda.set_device(0)
    t0 = time.time()
    lo_c, hi_c = (int(x) for x in args.member_cells.split(","))
    seq_stream = torch.cuda.Stream()
    streams, states, seq_states, cells, cu, Ms, alg = [], [], [], 0, 0, [], 0.0
    for i in range(args.members):
        s = scenario.ensemble_member(i, n_min=lo_c, n_max=hi_c)
        mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
        fz = s.forcing
        vt = list(fz.vortex) + [float(np.mean(s.fVertex))] if fz.vortex is not None else None

        def params(stream):
            return fb.make_params(s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                                  rho0=fz.rho0, rho_air=fz.rho_air, vortex=vt, precision=fb.FP32_TENDENCY,
                                  use_graph=True, stream=stream.cuda_stream)
        streams.append(torch.cuda.Stream())
        states.append(fb.state_init(mesh, params(streams[-1]), s.h0, s.u0, s.bottom))
        seq_states.append(fb.state_init(mesh, params(seq_stream), s.h0, s.u0, s.bottom))
        cells += int(s.mesh.nCells)
        cu += int(mesh.info().cell_updates_per_step)
        alg += fb.state_step_bytes(states[-1])[0]
        Ms.append(int(s.M[0]))
        del s
    setup_s = time.time() - t0
    hbm, _ = peaks()
    join = torch.cuda.Stream()

    def concurrent_round():
        fork = torch.cuda.Event()
        fork.record(join)
        for st, x in zip(states, streams):
            x.wait_event(fork)
            fb.lts_advance(st, 1)
        for x in streams:
            e = torch.cuda.Event()
            e.record(x)
            join.wait_event(e)

    def timed(run, stream, k):
        """per-round event times (ms) of k rounds on `stream`"""
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        torch.cuda.synchronize()
        evs[0].record(stream)
        for r in range(k):
            run()
            evs[r + 1].record(stream)
        torch.cuda.synchronize()
        return [evs[r].elapsed_time(evs[r + 1]) for r in range(k)]

    # plain, concurrent streams
    for _ in range(args.warmup):
        concurrent_round()
    conc = timed(concurrent_round, join, args.steps)
    for st in states:
        fb.synchronize(st)

    # plain, sequential: one stream, one member's step after another
    def sequential_round():
        for st in seq_states:
            fb.lts_advance(st, 1)
    for _ in range(args.warmup):
        sequential_round()
    seq = timed(sequential_round, seq_stream, args.steps)
    for st in seq_states:
        fb.synchronize(st)
        fb.state_destroy(st)

    # batched: tuning rounds, warm-up, then timed rounds with events on the batch stream
    stream = torch.cuda.Stream()
    b = fb.batch_create(states, autotune=True, stream=stream.cuda_stream)
    fb.batch_advance(b, 13)
    fb.batch_advance(b, args.warmup)
    fb.batch_synchronize(b)
    with ClockSampler(0) as clk:
        lat = timed(lambda: fb.batch_advance(b, 1), stream, args.steps)
    fb.batch_synchronize(b)
    ms_round = sum(lat) / len(lat)
    info = fb.batch_info(b)
    value = cu / (ms_round / 1000.0)

    def form(ts, launches):
        ms = sum(ts) / len(ts)
        return {"value": cu / (ms / 1000.0), "ms_per_round": ms, "step_hbm_frac": alg / (ms / 1000.0) / 1e9 / hbm,
                "launches_per_round": launches, "timing": "CUDA events"}
    lat = sorted(lat)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_round, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-tendency/f64-state", "data": "synthetic",
        "config": {"workload": "ensemble", "members": args.members, "member_cells": [lo_c, hi_c], "cells": cells,
                   "cell_updates_per_round": cu, "M": Ms,
                   "description": "batched ensemble of periodic-in-y shelf channels of seeded sizes, "
                                  "seeded roughness and Holland vortex track, M in {2,4,8}; one round = one "
                                  "coarse step of every member", "parallelism": "single"},
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "alg_bytes_per_round": alg,
        "step_hbm_frac": alg / (ms_round / 1000.0) / 1e9 / hbm,
        "plain_concurrent": form(conc, int(info.member_launches_per_round)),
        "plain_sequential": form(seq, int(info.member_launches_per_round)),
        "batched_vs_plain_concurrent": (sum(conc) / len(conc)) / ms_round,
        "batched_vs_plain_sequential": (sum(seq) / len(seq)) / ms_round,
        "batch": {"mode": ("merged launches", "graph branches", "merged per group, groups as branches",
                           "merged per group of <= 4, groups as branches")[info.mode],
                  "groups": info.groups,
                  "launches_per_round": int(info.launches_per_round), "threads_per_block": info.threads_per_block,
                  "ctas_per_sm": info.ctas_per_sm, "tile_order": "largest first" if info.tile_order == 0 else "member",
                  "tuned": bool(info.tuned),
                  "candidates_ms": {("branches" if k == 12 else "%s/tpb%d/cta%d" % (
                      ("merged", "grouped", "grouped4")[k // 4], (128, 256)[(k // 2) % 2], (0, 8)[k % 2])):
                      round(float(info.candidate_ms[k]), 3) for k in range(info.n_candidates)}},
        "gpu_launches": int(info.launches_per_round * args.steps + args.members),
        "setup_s": setup_s,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    fb.batch_destroy(b)


def run_serve(args, rank):
    """Serving loop: Poisson arrivals (rate --serve-rate per s, --serve-seconds
    of arrivals) of storm-surge requests, each on the resident 512x512 shelf
    channel or the 2.03M-cell basin (50/50), with a seeded vortex track and a
    duration drawn from 1-48 simulated hours times --serve-hours-scale, under a
    --serve-budget-gb HBM budget (fblts_server_*, FP32-tendency).  The same
    request stream is also served one request at a time (the plain form)."""
    if rank != 0:
        return
    import torch
    import paper_2405_10505_gb300 as fb
    from synth import scenario, basin
    torch.cuda.set_device(0)
    t_setup = time.time()
    shelf = scenario.shelf_case(vortex=True)
    bas = basin.basin_case()
    kinds = []
    for s in (shelf, bas):
        mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
        kinds.append((s, mesh, int(mesh.info().cell_updates_per_step)))
    setup_s = time.time() - t_setup
    rng = np.random.default_rng(2405)
    reqs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / args.serve_rate)
        if t > args.serve_seconds:
            break
        k = int(rng.integers(0, 2))
        s = kinds[k][0]
        hours = float(rng.uniform(1.0, 48.0)) * args.serve_hours_scale
        n = max(1, int(round(hours * 3600.0 / s.dt)))
        v = list(s.forcing.vortex)
        v[4] += float(rng.uniform(-0.1, 0.1)) * 1e6          # track origin and heading vary per request
        v[5] += float(rng.uniform(-0.1, 0.1)) * 1e6
        v[7] = float(rng.uniform(-2.0, 2.0))
        reqs.append((t, k, n, v))

    def serve(max_active):
        srv = fb.server_create(hbm_budget=int(args.serve_budget_gb * 1e9), max_active=max_active,
                               steps_per_issue=2)
        ids, pending, done, failed = [], list(reqs), 0, []
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while pending and pending[0][0] <= now:
                _, k, n, v = pending.pop(0)
                s, mesh, _ = kinds[k]
                fz = s.forcing
                p = fb.make_params(s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                                   rho0=fz.rho0, rho_air=fz.rho_air, vortex=v + [float(np.mean(s.fVertex))],
                                   precision=fb.FP32_TENDENCY)
                ids.append((fb.server_submit(srv, mesh, p, s.h0, s.u0, s.bottom, n), k, n))
            if fb.server_progress(srv):
                for rid, _, _ in ids:
                    status = fb.server_request_info(srv, rid).status
                    if status in (fb.REQ_DONE, fb.REQ_FAILED):
                        try:
                            fb.server_take(srv, rid, read=True)
                        except fb.FbltsError:
                            failed.append(rid)
                        done += 1
            elif not pending and done < len(reqs):
                time.sleep(0.0005)
        wall = time.perf_counter() - t0
        st = fb.server_stats(srv)
        lat = sorted(fb.server_request_info(srv, rid).t_done - fb.server_request_info(srv, rid).t_submit
                     for rid, _, _ in ids)
        cu = sum(kinds[k][2] * n for _, k, n in ids)
        fb.server_destroy(srv)
        return {"value": cu / wall, "wall_s": wall, "requests": len(ids), "failed": len(failed),
                "latency_s": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
                "max_running": int(st.max_running), "peak_device_gb": st.device_bytes_peak / 1e9}

    with ClockSampler(0) as clk:
        served = serve(args.serve_max_active)
    plain = serve(1)
    line = {
        "metric": METRIC, "value": served["value"], "unit": UNIT, "n_gpus": 1, "steps": served["requests"],
        "warmup": 0, "ms_per_step": 1000.0 * served["wall_s"] / max(1, served["requests"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-tendency/f64-state", "data": "synthetic",
        "config": {"workload": "serve", "rate_per_s": args.serve_rate, "arrival_window_s": args.serve_seconds,
                   "max_active": args.serve_max_active,
                   "hours_scale": args.serve_hours_scale, "budget_gb": args.serve_budget_gb,
                   "meshes": ["shelf 512x512 (262k cells, M=4)", "basin (2.03M cells, 3 levels, M=8)"],
                   "description": "Poisson arrivals of storm-surge requests, 50/50 on the two resident meshes, "
                                  "seeded vortex tracks, durations U[1,48] simulated hours x hours_scale; "
                                  "value = cell-updates/s over the run", "parallelism": "single"},
        "served": served, "plain_one_at_a_time": plain, "served_vs_plain": served["value"] / plain["value"],
        "latency_ms": {"p50": 1000.0 * served["latency_s"]["p50"], "p99": 1000.0 * served["latency_s"]["p99"]},
        "setup_s": setup_s, "clocks": clk.summary(),
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000, help="timed coarse steps (latency percentiles over them)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--latency-steps", type=int, default=1000,
                    help="coarse steps of the latency window (p50/p99), at least --steps")
    ap.add_argument("--impl", default="fblts", choices=["fblts", "reference"])
    ap.add_argument("--workload", default="basin")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="oracle instances for the CPU legs (default: one per host core)")
    ap.add_argument("--members", type=int, default=48, help="ensemble workload: members")
    ap.add_argument("--member-cells", default="20000,800000",
                    help="ensemble workload: range of member sizes (cells), lo,hi")
    ap.add_argument("--serve-rate", type=float, default=4.0, help="serve workload: arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serve workload: arrival window (s)")
    ap.add_argument("--serve-hours-scale", type=float, default=0.01,
                    help="serve workload: factor on the 1-48 h durations")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0, help="serve workload: HBM budget (GB)")
    ap.add_argument("--serve-max-active", type=int, default=6,
                    help="serve workload: running requests at once (0 = as many as the budget allows)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other-precision and global FB-RK(3,2) comparison runs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "ensemble" and args.impl != "reference":
        run_ensemble(args, rank)
        return
    if args.workload == "serve" and args.impl != "reference":
        run_serve(args, rank)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return
    s, desc = make_workload(args.workload)

    import torch
    import paper_2405_10505_gb300 as fb
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prec = fb.FP64 if args.precision == "fp64" else fb.FP32_TENDENCY
    stream = torch.cuda.Stream()
    mesh = fb.mesh_create(s.mesh, s.fVertex, level=s.level, M=s.M)
    fz = s.forcing
    vt = list(fz.vortex) + [float(np.mean(s.fVertex))] if fz.vortex is not None else None
    params = fb.make_params(s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                            rho0=fz.rho0, rho_air=fz.rho_air, vortex=vt, precision=prec,
                            stream=stream.cuda_stream, use_graph=True)
    st = fb.state_init(mesh, params, s.h0, s.u0, s.bottom)
    info = mesh.info()
    cu = int(info.cell_updates_per_step)
    launches = fb.launches_per_step(st)
    step_bytes, _ = fb.state_step_bytes(st)
    moved_step = sum(v[1] for v in fb.state_bytes_by_kind(st).values())

    fb.lts_advance(st, args.warmup)
    fb.synchronize(st)

    # timed region: K coarse steps, one event per step for the latency percentiles
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs[0].record(stream)
        for k in range(args.steps):
            fb.lts_advance(st, 1)
            evs[k + 1].record(stream)
        fb.synchronize(st)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms_total = evs[0].elapsed_time(evs[-1])
    lat = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps))
    if dist:
        ms_total = max_over_ranks(ms_total, dist, torch, "cuda")
    ms_step = ms_total / args.steps
    value = replica_value(world, cu, args.steps, ms_total)

    # latency percentiles over a window of at least 1000 coarse steps (after the
    # timed region, whatever --steps is), one event pair per step
    n_lat = max(args.latency_steps, args.steps)
    if n_lat > args.steps:
        levs = [torch.cuda.Event(enable_timing=True) for _ in range(n_lat + 1)]
        levs[0].record(stream)
        for k in range(n_lat):
            fb.lts_advance(st, 1)
            levs[k + 1].record(stream)
        fb.synchronize(st)
        lat = sorted(levs[k].elapsed_time(levs[k + 1]) for k in range(n_lat))

    # per-kernel profile (launch by launch with events on the same stream)
    prof = fb.state_profile_step(st)
    bykind = fb.state_bytes_by_kind(st)
    dom = max(prof, key=lambda k: prof[k][0])
    dms, dn, dbytes = prof[dom]
    dmoved = bykind[dom][1]
    hbm, peak_src = peaks()
    achieved = dbytes / (dms / 1000.0) / 1e9
    kernel_name = {"cell": "cell_pass", "vertex": "vert_pass", "edge_prep": "eprep_pass",
                   "edge": "edge_pass", "trisk": "trisk_pass"}.get(dom, dom)
    traffic = traffic_for(args.workload, args.precision, kernel_name)

    # end to end through the public host-buffer call: H2D inputs, 1 step, D2H result
    nC, nE = info.nCells, info.nEdges
    hin = torch.empty(nC, dtype=torch.float64, pin_memory=True).numpy()
    uin = torch.empty(nE, dtype=torch.float64, pin_memory=True).numpy()
    hout = torch.empty(nC, dtype=torch.float64, pin_memory=True).numpy()
    uout = torch.empty(nE, dtype=torch.float64, pin_memory=True).numpy()
    fb.state_read(st, hin, uin)
    n_e2e = max(3, min(args.steps, 20))
    fb.run_host(st, hin, uin, 1, hout, uout)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        fb.run_host(st, hin, uin, 1, hout, uout)
    e2e_s = time.perf_counter() - t0
    e2e_v = world * cu * n_e2e / e2e_s

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == fb.FP64 else "f32-tendency/f64-state",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "cells": nC, "edges": nE,
                   "vertices": int(info.nVertices), "levels": int(info.nLevels), "M": list(s.M),
                   "cells_per_level": [int(x) for x in list(info.cells_per_level)[: info.nLevels]],
                   "cell_updates_per_step": cu, "precision": args.precision,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs larger than L2: {step_bytes / 1e6:.0f} MB algorithmic traffic per step"},
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "steps": len(lat)},
        "alg_bytes_per_step": step_bytes,
        "alg_bytes_per_cell_update": step_bytes / cu,
        "moved_bytes_per_step": moved_step,
        "step_hbm_frac": step_bytes / (ms_step / 1000.0) / 1e9 / hbm,
        "step_moved_frac": moved_step / (ms_step / 1000.0) / 1e9 / hbm,
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src,
                     "alg_bytes_per_launch": dbytes / max(dn, 1), "moved_bytes_per_launch": dmoved / max(dn, 1),
                     "moved_frac": dmoved / (dms / 1000.0) / 1e9 / hbm,
                     "moved_over_alg": dmoved / dbytes if dbytes else None,
                     "traffic_over_alg": (traffic / (dbytes / max(dn, 1))) if (traffic and dbytes) else None,
                     "launches_per_step": dn, "share_of_step": dms / sum(v[0] for v in prof.values())},
        "profile_ms_per_step": {k: round(v[0], 4) for k, v in prof.items()},
        "bytes_per_step_by_kind": {k: {"alg": v[0], "moved": v[1]} for k, v in bykind.items() if v[1] > 0},
        "gpu_launches": int(launches * args.steps + 1),
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": 8 * (nC + nE),
                "d2h_bytes_per_step": 8 * (nC + nE), "steps": n_e2e},
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_variants:
        # the same workload in the other precision (fewer timed steps)
        oprec = fb.FP64 if prec == fb.FP32_TENDENCY else fb.FP32_TENDENCY
        ost = fb.state_init(mesh, fb.make_params(
            s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd, rho0=fz.rho0,
            rho_air=fz.rho_air, vortex=vt, precision=oprec, stream=stream.cuda_stream, use_graph=True),
            s.h0, s.u0, s.bottom)
        k2 = max(3, min(args.steps, 10))
        oms = timed_steps(fb, torch, ost, stream, 3, k2)
        line["other_precision"] = {"precision": "fp64" if oprec == fb.FP64 else "fp32",
                                   "value": cu / (oms / 1000.0), "ms_per_step": oms, "steps": k2}
        fb.state_destroy(ost)
        # the fast/slow operator splitting of Sec. 3.2 (first order in time), same precision
        sst = fb.state_init(mesh, fb.make_params(
            s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd, rho0=fz.rho0,
            rho_air=fz.rho_air, vortex=vt, precision=prec, stream=stream.cuda_stream, use_graph=True, split=True),
            s.h0, s.u0, s.bottom)
        sms = timed_steps(fb, torch, sst, stream, 3, max(3, min(args.steps, 20)))
        sb, _ = fb.state_step_bytes(sst)
        line["split"] = {"value": cu / (sms / 1000.0), "ms_per_step": sms, "speedup_vs_unsplit": ms_step / sms,
                         "alg_bytes_per_step": sb, "step_hbm_frac": sb / (sms / 1000.0) / 1e9 / hbm}
        fb.state_destroy(sst)
        # its variant with the slow terms of every finer level evaluated once per
        # step of that level (proposed at the end of Sec. 4.2)
        if int(info.nLevels) > 1:
            sst = fb.state_init(mesh, fb.make_params(
                s.dt, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd, rho0=fz.rho0,
                rho_air=fz.rho_air, vortex=vt, precision=prec, stream=stream.cuda_stream, use_graph=True, split=2),
                s.h0, s.u0, s.bottom)
            fms = timed_steps(fb, torch, sst, stream, 3, max(3, min(args.steps, 20)))
            line["split_per_level_step"] = {"value": cu / (fms / 1000.0), "ms_per_step": fms,
                                            "speedup_vs_unsplit": ms_step / fms}
            fb.state_destroy(sst)
        # global FB-RK(3,2) at the finest level's step on the same mesh (no LTS):
        # the time one coarse step's simulated interval takes without local time stepping
        nl = int(info.nLevels)
        if nl > 1:
            ratio = int(np.prod(s.M))
            gmesh = fb.mesh_create(s.mesh, s.fVertex, level=np.zeros(nC, np.int32), M=[])
            gst = fb.state_init(gmesh, fb.make_params(
                s.dt / ratio, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                rho0=fz.rho0, rho_air=fz.rho_air, vortex=vt, precision=prec, stream=stream.cuda_stream,
                use_graph=True), s.h0, s.u0, s.bottom)
            kg = ratio * max(2, min(args.steps // 20, 5))
            gms = timed_steps(fb, torch, gst, stream, ratio, kg)
            line["global_fbrk"] = {
                "dt": s.dt / ratio, "steps": kg, "ms_per_step": gms,
                "ms_per_coarse_interval": gms * ratio,
                "cell_updates_per_s": nC / (gms / 1000.0),
                "lts_speedup": gms * ratio / ms_step}
            fb.state_destroy(gst)
            # classical RK4 (the paper's comparison integrator, Sec. 4.2, Tab. 2) on the
            # same one-level mesh, at the finest step scaled by the ratio of the two
            # schemes' linear gravity-wave stability limits
            rk_ratio = RK4_IMAG_LIMIT / fbrk32_imag_limit(fb.PAPER_BETA)
            dt_rk = s.dt / ratio * rk_ratio
            rst = fb.state_init(gmesh, fb.make_params(
                dt_rk, g=s.g, forcing=forcing_flags(s), wind=(fz.wind_u, fz.wind_v), cd=fz.cd,
                rho0=fz.rho0, rho_air=fz.rho_air, vortex=vt, precision=prec, stream=stream.cuda_stream,
                use_graph=True, scheme=fb.SCHEME_RK4), s.h0, s.u0, s.bottom)
            kr = max(10, min(args.steps, 50))
            rms = timed_steps(fb, torch, rst, stream, 3, kr)
            per_interval = rms * s.dt / dt_rk
            rb, _ = fb.state_step_bytes(rst)
            line["global_rk4"] = {
                "dt": dt_rk, "dt_over_fbrk32_dt": rk_ratio, "steps": kr, "ms_per_step": rms,
                "ms_per_coarse_interval": per_interval, "cell_updates_per_s": nC / (rms / 1000.0),
                "step_hbm_frac": rb / (rms / 1000.0) / 1e9 / hbm,
                "lts_speedup": per_interval / ms_step, "split_lts_speedup": per_interval / sms}
            fb.state_destroy(rst)
            fb.mesh_destroy(gmesh)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle timed on a bounded sample (whole coarse steps of the workload, or of
        # its 1/64-length sample for the basin), one instance per host core
        T = cpu_threads(args)
        ts, tname = reference_sample(args.workload) if args.workload == "basin" else (s, args.workload)
        nt, el, _, _, _ = oracle_sample(ts, budget_s=3.0, threads=T)
        line["cpu_baseline"] = {"value": cell_updates_per_step(ts) * nt / el, "unit": UNIT, "cores": T,
                                "kind": "oracle",
                                "sample": f"{nt} whole coarse steps of {tname} in {el:.1f} s over {T} threads "
                                          "(one single-threaded C oracle instance per host core, each on its own "
                                          "copy of the state)",
                                "host_cores_available": os.cpu_count()}
        # the error of this path against the oracle on whole coarse steps of the
        # workload, or of its 1/8-length sample (same recipe) for the basin
        ws, sample_name = s, args.workload
        if args.workload == "basin":
            ws, _ = make_workload("basin_small")
            sample_name = "basin_small (1/8-length sample of the basin: same recipe, Ly 1200 km)"
        _, _, ho, uo, n = oracle_sample(ws)
        wmesh = mesh if ws is s else fb.mesh_create(ws.mesh, ws.fVertex, level=ws.level, M=ws.M)
        wfz = ws.forcing
        wvt = list(wfz.vortex) + [float(np.mean(ws.fVertex))] if wfz.vortex is not None else None
        wparams = fb.make_params(ws.dt, g=ws.g, forcing=forcing_flags(ws), wind=(wfz.wind_u, wfz.wind_v),
                                 cd=wfz.cd, rho0=wfz.rho0, rho_air=wfz.rho_air, vortex=wvt, precision=prec,
                                 stream=stream.cuda_stream, use_graph=True)
        errs = {}
        for pname, pv in (("fp32", fb.FP32_TENDENCY), ("fp64", fb.FP64)):
            wparams.precision = pv
            st2 = fb.state_init(wmesh, wparams, ws.h0, ws.u0, ws.bottom)
            fb.lts_advance(st2, n)
            h, u = fb.state_read(st2)
            fb.state_destroy(st2)
            errs[pname] = {"h_rel_max": float(np.max(np.abs(h - ho) / np.abs(ho))),
                           "u_rel_max": float(np.max(np.abs(u - uo)) / max(np.max(np.abs(uo)), 1e-300))}
        if not args.no_variants:
            # the split FP32 path against the split oracle on the same window
            import oracle as orc
            hs_o, us_o = orc.fblts(orc.Mesh.from_scenario(ws), orc.scenario_params(ws, split=True), ws.level, ws.M,
                                   ws.h0, ws.u0, ws.dt, n)
            wparams.precision = fb.FP32_TENDENCY
            wparams.split = 1
            st2 = fb.state_init(wmesh, wparams, ws.h0, ws.u0, ws.bottom)
            fb.lts_advance(st2, n)
            h, u = fb.state_read(st2)
            fb.state_destroy(st2)
            errs["fp32_split"] = {"h_rel_max": float(np.max(np.abs(h - hs_o) / np.abs(hs_o))),
                                  "u_rel_max": float(np.max(np.abs(u - us_o)) / max(np.max(np.abs(us_o)), 1e-300)),
                                  "vs": "split oracle"}
        line["err_vs_oracle"] = {"workload": sample_name, "coarse_steps": n, **errs}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
