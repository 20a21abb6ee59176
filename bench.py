#!/usr/bin/env python3
"""Benchmark of the hybrid tree force path on GB300.

One step = one soft step dt_s of the hybrid scheme (n_hard hard sub-steps,
each with a tree rebuild and the hard force, plus the soft force at the last
one) for one Plummer sphere of N = 2^17 particles (seed 1, eps = 1/128,
theta = 0.5, R1 = 4 eps, R2 = 8 eps, dt_s = 1/128, n_hard = 4), FP32 pair
kernels on FP64 state. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--gpus N > 1 runs N independent replicas (torchrun, one rank per GPU); the
path has no exchange step, so there is no collective on the data path.
--impl reference times the CPU FP64 oracle on the host cores instead.
Beside the headline the line carries the same workload with reused trees and
neighbour lists (a Verlet skin; not the paper's scheme) and two compact
sub-records measured in the same run: "large" (one Hernquist sphere of 2^24
particles, theta = 0.4, n_hard = 8) and "batched" (512 Plummer spheres of
uneven N in one call per step, against the same systems one per call in
FP64). Each workload also runs alone: --workload large | batched | served |
paper (hybrid against normal tree with the paper's parameter set).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 1 << 17
METRIC = "particle-steps/s"
FLOPS_PER_INTERACTION = 20          # monopole pair: 3 sub, 3 fma, rsqrt, 3 mul, 3 fma (by convention 20)
# DRAM bytes (read + write) of one far-pair launch on this workload, from one ncu capture of the current far
# kernel for each variant the keys name (n_crit, threads per group, staging depth). Reported as the roofline's
# traffic only when the autotuner picks one of these variants, else None.
FAR_TRAFFIC_BYTES = {(128, 32, 2): 57.37e6, (128, 32, 4): 57.31e6}
CLOCK_INTERVAL_MS = 20
L2_FLUSH_BYTES = 256 << 20
ENERGY_MAX_N = 1 << 18              # largest N whose energy the paper comparison evaluates (O(N^2) FP64)
# Verlet skin of the reused-list measurement: twice the distance the fastest particle of the Plummer sphere
# (escape speed sqrt(2) at the centre, G = M = a = 1) covers in the three drifts that reuse a build's lists
# (3/512 each), rounded up: 2 x 1.42 x 3/512 = 0.0166 -> 0.025. Steps that exceed it rebuild by themselves.
REUSE_SKIN = 0.025


def workload(n):
    eps = 1.0 / 128
    return dict(n=n, seed=1, eps=eps, theta=0.5, R1=4 * eps, R2=8 * eps, dt_soft=1.0 / 128, n_hard=4,
                n_leaf=16, n_crit=64)


def workload_name(w):
    return ("Plummer sphere N=%d seed %d, eps=1/128, theta=0.5, R1=4eps, R2=8eps, dt_s=1/128, n_hard=4; "
            "FP32 pair kernels on group-relative coordinates, FP64 state" % (w["n"], w["seed"]))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def job_rate(units_per_rank, seconds, dist=None, device="cuda"):
    """Whole-job throughput of independent replicas: the units of all ranks over the slowest rank's time
    (max over ranks). Returns (rate, max seconds)."""
    if dist is None:
        return units_per_rank / seconds, seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return dist.get_world_size() * units_per_rank / tmax, tmax


def fp32_peak_tflops(nsm, sm_mhz):
    # 128 FP32 lanes per SM, 2 flops per FMA
    return nsm * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(CLOCK_INTERVAL_MS)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "interval_ms": CLOCK_INTERVAL_MS}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return out
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        out.update(sm_mhz=sm[len(sm) // 2] if sm else None, sm_max_mhz=max(mx) if mx else None, reasons=reasons,
                   samples=len(rows))
        return out


def force_error_rms(state, a_s, a_h, eps, nsample=512, seed=0):
    """rms over sampled sinks of |a_gpu - a_direct| / |a_direct| (direct FP64 summation, CPU)."""
    import numpy as np
    import oracle
    n = len(state["x"])
    rng = np.random.default_rng(seed)
    sink = np.sort(rng.choice(n, min(nsample, n), replace=False))
    full, _ = oracle.direct(state["x"], state["y"], state["z"], state["m"], eps=eps, sinks=sink)
    a = (a_s + a_h)[sink]
    e = np.linalg.norm(a - full, axis=1) / np.linalg.norm(full, axis=1)
    return float(np.sqrt(np.mean(e * e)))


def cpu_baseline(w, max_seconds=20.0):
    """The oracle as it stands, on this host's cores: whole hybrid steps of the same workload."""
    import numpy as np
    import oracle
    from paper_1406_6158_gb300 import ics
    st = ics.plummer(w["n"], w["seed"])
    p = oracle.Params(eps=w["eps"], theta=w["theta"], R1=w["R1"], R2=w["R2"], dt_soft=w["dt_soft"],
                      n_hard=w["n_hard"], n_leaf=w["n_leaf"], n_crit=w["n_crit"])
    a_s, a_h = oracle.forces(st, p)
    steps, t = 0, 0.0
    while t < max_seconds and steps < 64:
        t0 = time.perf_counter()
        a_s, a_h = oracle.hybrid_steps(st, p, 1, a_s, a_h)
        t += time.perf_counter() - t0
        steps += 1
    return {"value": w["n"] * steps / t, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d whole soft step(s) of the same workload (N=%d), FP64, OpenMP over sink groups" %
                      (steps, w["n"]), "seconds": t}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import numpy as np
    from paper_1406_6158_gb300 import ics
    st = ics.plummer(w["n"], w["seed"])
    p = oracle.Params(eps=w["eps"], theta=w["theta"], R1=w["R1"], R2=w["R2"], dt_soft=w["dt_soft"],
                      n_hard=w["n_hard"], n_leaf=w["n_leaf"], n_crit=w["n_crit"])
    a_s, a_h = oracle.forces(st, p)
    for _ in range(min(args.warmup, 3)):
        a_s, a_h = oracle.hybrid_steps(st, p, 1, a_s, a_h)
    # whole soft steps of the workload, at most args.steps of them and as many as fit in the time box, so that
    # the run ends within a few minutes (one soft step of the oracle takes most of a second here)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps and (done == 0 or time.perf_counter() - t0 < args.ref_max_seconds):
        a_s, a_h = oracle.hybrid_steps(st, p, 1, a_s, a_h)
        done += 1
    t = time.perf_counter() - t0
    v = w["n"] * done / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "steps_timed": done, "warmup": args.warmup, "ms_per_step": 1e3 * t / done, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "N": w["n"], "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "%d whole soft steps of the workload (of %d asked, time box %.0f s) after %d "
                                   "warm-up steps" % (done, args.steps, args.ref_max_seconds,
                                                      min(args.warmup, 3))},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def c4_systems(count=512, seed=3):
    """The batched ensemble: `count` Plummer spheres, N log-uniform in [2^10, 2^17], eps = 1/(4 N^(1/3))."""
    from paper_1406_6158_gb300 import ics
    sizes = ics.ensemble_sizes(count, 10.0, 17.0, seed)
    out = []
    for k, n in enumerate(sizes):
        eps = 1.0 / (4.0 * float(n) ** (1.0 / 3.0))
        out.append((int(n), seed * 1000003 + k, dict(eps=eps, theta=0.5, R1=4 * eps, R2=8 * eps, dt_soft=1.0 / 128)))
    return out


C4_NAME = ("batched ensemble: %d Plummer spheres, N log-uniform in [2^10, 2^17] (seed 3), total N=%d, "
           "eps=1/(4 N^(1/3)), theta=0.5, R1=4eps, R2=8eps, dt_s=1/128, n_hard=4; one call per step for all "
           "systems (CUDA graph), FP32 pairs, FP64 state")


def c4_record(args, steps, warmup):
    """Batched FP32 form (one call advances all systems; autotuned n_crit, threads per group, staging depth)
    against the plain form (FP64, one system per call), same systems, one soft step each."""
    import numpy as np
    import torch
    from paper_1406_6158_gb300 import hybrid, ics
    specs = c4_systems(args.c4_count)
    total = sum(n for n, _, _ in specs)
    states = [ics.plummer(n, sd) for n, sd, _ in specs]
    base = dict(n_hard=4, n_leaf=16, n_crit=64)

    def per(prec, kw):
        return hybrid.Params(precision=prec, **base, **kw)

    stream = torch.cuda.Stream()           # a stream of its own: the library replays captured CUDA graphs on it
    torch.cuda.set_stream(stream)
    # ---- batched FP32 ----
    ctx = hybrid.Context(per(1, specs[0][2]), stream)
    sysb = [hybrid.System(st, precision=1, ids=False, params=per(1, kw)) for st, (_, _, kw) in zip(states, specs)]
    chosen, table = ctx.hybrid_autotune(sysb)
    ctx.hybrid_step_batched(sysb, 0)
    for _ in range(warmup):
        ctx.hybrid_step_batched(sysb, 1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(torch.cuda.current_device())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = ctx.hybrid_launch_count()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.hybrid_step_batched(sysb, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ctx.hybrid_launch_count() - launches0
    t_b = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    v_b = total * steps / t_b
    # ---- plain FP64, one system per call ----
    ctx64 = hybrid.Context(per(0, specs[0][2]), stream)
    sys64 = [hybrid.System(st, precision=0, ids=False, params=per(0, kw)) for st, (_, _, kw) in zip(states, specs)]
    for s in sys64:
        ctx64.hybrid_step(s, 0)
    torch.cuda.synchronize()
    clocks64 = ClockSampler(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks64.start()
    e0.record(stream)
    for s in sys64:
        ctx64.hybrid_step(s, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    clk64 = clocks64.stop()
    t_p = e0.elapsed_time(e1) / 1e3
    v_p = total / t_p
    # ---- force error against direct summation on a few systems ----
    rng = np.random.default_rng(7)
    pick = sorted(rng.choice(len(specs), 4, replace=False))
    errs = {"fp32_batched": [], "fp64_plain": []}
    for k in pick:
        for name, sysl in (("fp32_batched", sysb), ("fp64_plain", sys64)):
            out = sysl[k].numpy()
            a_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)
            a_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)
            errs[name].append(force_error_rms(out, a_s, a_h, specs[k][2]["eps"], nsample=256))
    ctx.close()
    ctx64.close()
    del sysb, sys64, flush
    torch.cuda.empty_cache()
    return {
        "workload": C4_NAME % (len(specs), total), "N_total": total, "systems": len(specs),
        "metric": METRIC, "value": v_b, "unit": METRIC, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_b / steps, "dtype": "f32", "l2": "flushed (256 MiB write) before every timed step",
        "autotune": {"chosen": {"n_crit": chosen[0], "threads_per_group": chosen[1], "tile_depth": chosen[2]},
                     "est_ms_per_step": [round(float(x), 3) for x in table]},
        "plain_fp64": {"value": v_p, "unit": METRIC, "ms_per_step": 1e3 * t_p, "clocks": clk64,
                       "form": "FP64 pairs, one system per hybrid_step call, same systems"},
        "batched_over_plain": v_b / v_p,
        "force_err_rms_vs_direct": {k: float(np.mean(v)) for k, v in errs.items()},
        "gpu_launches": launches, "clocks": clk,
    }


def run_c4(args):
    from paper_1406_6158_gb300 import build as cuda_build
    cuda_build.build()
    r = c4_record(args, args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": 1, "steps": r["steps"],
        "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "N_total": r["N_total"], "systems": r["systems"], "l2": r["l2"]},
    }
    line.update({k: r[k] for k in ("autotune", "plain_fp64", "batched_over_plain", "force_err_rms_vs_direct",
                                   "gpu_launches", "clocks")})
    print(json.dumps(line), flush=True)
    return 0


def c5_trace(count, seed=5, rate=200.0):
    """Served stream: Poisson arrivals at `rate` per second, N log-uniform in [2^12, 2^21], 32 soft steps."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    sizes = np.floor(2.0 ** rng.uniform(12.0, 21.0, count)).astype(np.int64)
    return arrivals, sizes


def run_c5(args):
    """Continuous batching (hybrid_server_*, FP32 form) on a Poisson request trace, wall-clock driven:
    latency = completion - arrival per request; beside it the plain FP64 form serving the same trace
    one request at a time (FIFO), from its measured per-request step rate."""
    import numpy as np
    import torch
    from paper_1406_6158_gb300 import build as cuda_build
    from paper_1406_6158_gb300 import hybrid, ics
    cuda_build.build()
    count, steps = args.c5_count, 32
    arrivals, sizes = c5_trace(count)
    tic = time.perf_counter()
    states = [ics.plummer(int(n), 5 * 1000003 + k) for k, n in enumerate(sizes)]
    log = (lambda *a: print("[served %.1fs]" % (time.perf_counter() - tic), *a, file=sys.stderr, flush=True)) \
        if args.verbose else (lambda *a: None)
    log("initial conditions ready: %d requests, %d particles" % (count, int(sizes.sum())))

    def rparams(n, prec):
        eps = 1.0 / (4.0 * float(n) ** (1.0 / 3.0))
        return hybrid.Params(eps=eps, theta=0.5, R1=4 * eps, R2=8 * eps, dt_soft=1.0 / 128, n_hard=4,
                             n_leaf=16, n_crit=128, threads_per_group=32, precision=prec)

    budget = 150e9
    torch.cuda.set_stream(torch.cuda.Stream())   # a stream of its own: captured CUDA graphs are replayed on it
    srv = hybrid.Server(rparams(1 << 16, 1), budget)
    # warm-up: one small request through the server (module load, first graph capture)
    srv.submit(count, ics.plummer(4096, 1), rparams(4096, 1), 2)
    while srv.next() is None:
        srv.step()
    log("warm-up done")
    done, lat, k = 0, np.zeros(count), 0
    busy_steps = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_first = None
    while done < count:
        now = time.perf_counter() - t0
        while k < count and arrivals[k] <= now:
            srv.submit(k, states[k], rparams(sizes[k], 1), steps)
            k += 1
        a, q, f = srv.step()
        if a == 0 and q == 0 and f == 0:
            if k < count:
                time.sleep(max(0.0, arrivals[k] - (time.perf_counter() - t0)))
            continue
        busy_steps += 1
        if busy_steps % 20 == 0:
            log("step %d: active %d queued %d finished %d done %d submitted %d, %.1f GB charged"
                % (busy_steps, a, q, f, done, k, srv.used_bytes() / 1e9))
        if time.perf_counter() - t0 > args.c5_max_seconds:
            raise RuntimeError("served stream exceeded %.0f s" % args.c5_max_seconds)
        if t_first is None:
            t_first = now
        while True:
            r = srv.next()
            if r is None:
                break
            lat[r[0]] = (time.perf_counter() - t0) - arrivals[r[0]]
            done += 1
    t_end = time.perf_counter() - t0
    srv.close()
    log("served: %.1f s, %d server steps" % (t_end, busy_steps))
    work = float(sizes.sum()) * steps
    served = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
              "mean_s": float(lat.mean()), "throughput": work / (t_end - arrivals[0]),
              "server_steps": busy_steps}
    # plain FP64, one request at a time: measured step rate of sampled requests, FIFO queue over the trace
    ctx64 = hybrid.Context(rparams(1 << 16, 0))
    rates = []
    for j in np.linspace(0, count - 1, 3).astype(int):
        s64 = hybrid.System(states[j], precision=0, ids=False, params=rparams(sizes[j], 0))
        ctx64.hybrid_step(s64, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx64.hybrid_step(s64, 1)
        e1.record()
        torch.cuda.synchronize()
        rates.append(float(sizes[j]) / (e0.elapsed_time(e1) / 1e3))
        log("FP64 sample N=%d: %.3g particle-steps/s" % (sizes[j], rates[-1]))
    ctx64.close()
    rate64 = float(np.mean(rates))
    t_free, lat64 = 0.0, np.zeros(count)
    for i in range(count):
        start = max(t_free, arrivals[i])
        t_free = start + float(sizes[i]) * steps / rate64
        lat64[i] = t_free - arrivals[i]
    line = {
        "metric": "served p50/p99 latency and particle-steps/s", "value": served["throughput"],
        "unit": METRIC, "n_gpus": 1, "steps": steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "served stream: first %d requests of a Poisson trace at 200 req/s (seed 5), "
                               "Plummer spheres with N log-uniform in [2^12, 2^21], 32 soft steps each, "
                               "eps=1/(4 N^(1/3)), theta=0.5, R1=4eps, R2=8eps, dt_s=1/128, n_hard=4; "
                               "admission by %d B per particle under a 150 GB budget; FP32 pairs, FP64 state"
                               % (count, hybrid.SERVER_BYTES_PER_PARTICLE),
                   "requests": count, "particles_total": int(sizes.sum()),
                   "offered_particle_steps_per_s": work / float(arrivals[-1] - arrivals[0] + 1e-9)},
        "served": served,
        "serial_plain_fp64": {"p50_s": float(np.percentile(lat64, 50)), "p99_s": float(np.percentile(lat64, 99)),
                              "throughput": rate64,
                              "basis": "FP64 soft-step rate measured on 3 requests of the trace; FIFO, one "
                                       "request at a time"},
    }
    print(json.dumps(line), flush=True)
    return 0


def hbm_stages(n, n_hard, ms, nodes=None):
    """Achieved HBM bandwidth of the memory-bound stages from their live times per soft step and their
    algorithmic bytes (n_hard builds and drift launches per soft step):
      sort        per particle 36 (keys: x, y, z in, key and index out) + 12 (key in, bucket out) + 24 (key and
                  bucket in, key and index out to the bucket) + 24 (key and index in and out of the bucket sort):
                  the sample sort the builds take between steps (a build that falls back to the radix sort moves
                  36 + 8 + 8 x 24; the line reports the fallbacks)
      topology    per particle 8 (sorted key in); per node 24 out (first, count, level, first child, children,
                  parent)
      moments     per particle 32 (FP32 hi/lo position copies in); per node 24 in (the topology) and 72 out (the
                  walk's and pair kernels' records: centre of mass and mass hi/lo, lo and B2, opening and
                  neighbour radii, topology)
      kick_drift  per particle 108 (v 24, a 12, x 24 in; v 24, x 24 out)
    nodes: tree nodes of one build (topology and moments are reported only when it is given)."""
    peak = float(measured_peaks().get("hbm_gbs", 6655.6))
    per = {"sort": (36 + 12 + 24 + 24, 0), "kick_drift": (108, 0)}
    if nodes:
        per["topology"] = (8, 24)
        per["moments"] = (32, 24 + 72)
    out = {}
    for name, (pp, pn) in per.items():
        t = ms.get(name)
        if not t:
            continue
        launch_bytes = n * pp + (nodes or 0) * pn
        gbs = launch_bytes * n_hard / (t / 1e3) / 1e9
        out[name] = {"bytes_per_launch": launch_bytes, "bytes_per_particle": pp, "bytes_per_node": pn,
                     "launches_per_step": n_hard, "GB/s": gbs, "frac_of_measured_hbm": gbs / peak}
    return out


C3_NAME = ("Hernquist sphere N=%d seed 2, a=1, r<=100, eps=1/512, theta=0.4, R1=3eps, R2=6eps, dt_s=1/128, "
           "n_hard=8; FP32 pairs, FP64 state")


def c3_cpu_leg(st, P, ngroups_sample=64):
    """The oracle on the host's cores for the large workload, sampled: one whole tree build (timed) and the
    soft and hard forces of sampled groups (timed), scaled to one soft step (n_hard builds, one soft and n_hard
    hard force evaluations over all groups)."""
    import numpy as np
    import oracle
    oracle.build()
    op = oracle.Params(G=P.G, eps=P.eps, theta=P.theta, R1=P.R1, R2=P.R2, dt_soft=P.dt_soft, a_err=P.a_err,
                       n_hard=P.n_hard, n_leaf=P.n_leaf, n_crit=P.n_crit, mac=P.mac)
    t0 = time.perf_counter()
    T = oracle.Tree(st["x"], st["y"], st["z"], st["m"], op)
    t_build = time.perf_counter() - t0
    sel = np.sort(np.random.default_rng(5).choice(T.ng, min(ngroups_sample, T.ng), replace=False))
    t0 = time.perf_counter()
    T.forces(groups=sel, mode=1)
    t_soft = (time.perf_counter() - t0) * T.ng / len(sel)
    t0 = time.perf_counter()
    T.forces(groups=sel, mode=2)
    t_hard = (time.perf_counter() - t0) * T.ng / len(sel)
    step = P.n_hard * t_build + t_soft + P.n_hard * t_hard
    n = len(st["x"])
    return {"value": n / step, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one tree build of all %d particles (%.1f s) and the soft and hard forces of %d of %d groups, "
                      "scaled to one soft step = %d builds + 1 soft + %d hard evaluations over all groups "
                      "(%.0f s estimated)" % (n, t_build, len(sel), T.ng, P.n_hard, P.n_hard, step)}


def c3_record(args, steps, warmup, with_cpu=True):
    """Large single system: Hernquist sphere N=2^24 (seed 2, a=1, r<=100), eps=1/512, theta=0.4, R1=3eps,
    R2=6eps, dt_s=1/128, n_hard=8, FP32 pairs on FP64 state."""
    import numpy as np
    import torch
    from paper_1406_6158_gb300 import hybrid, ics
    n = args.n if args.n != N_DEFAULT else 1 << 24
    eps = 1.0 / 512
    tic = time.perf_counter()
    st = ics.hernquist(n, 2)
    t_ic = time.perf_counter() - tic
    P = hybrid.Params(eps=eps, theta=0.4, R1=3 * eps, R2=6 * eps, dt_soft=1.0 / 128, n_hard=8, n_leaf=16,
                      n_crit=128, threads_per_group=32, precision=1)
    stream = torch.cuda.Stream()           # a stream of its own: the library replays captured CUDA graphs on it
    torch.cuda.set_stream(stream)
    ctx = hybrid.Context(P, stream)
    s = hybrid.System(st, precision=1, ids=False)
    if args.tune == "auto":
        cands = [(64, 16, 0), (128, 32, 0), (128, 32, 2), (128, 16, 0), (256, 64, 0), (256, 64, 2), (256, 32, 0),
                 (512, 128, 0), (512, 64, 0)]
    else:                                  # a fixed choice, e.g. to profile the autotuned configuration
        cands = [tuple(int(v) for v in args.tune.split(","))]
    chosen, _ = ctx.hybrid_autotune(s, cands)
    ctx.hybrid_step(s, 0)
    nodes, groups = ctx.tree_info()
    for _ in range(warmup):
        ctx.hybrid_step(s, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ctx.hybrid_profile(True)
    for k in range(9):
        ctx.hybrid_profile_read(k, reset=True)
    launches0 = ctx.hybrid_launch_count()
    fallbacks0 = ctx.hybrid_sort_fallbacks()
    clocks = ClockSampler(torch.cuda.current_device())
    inter_far = inter_near = 0
    torch.cuda.synchronize()
    clocks.start()
    for k in range(steps):
        ev[k][0].record(stream)
        ctx.hybrid_step(s, 1)
        ev[k][1].record(stream)
        fi, ni = ctx.hybrid_interactions()
        inter_far += fi
        inter_near += ni
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ctx.hybrid_launch_count() - launches0
    fallbacks = ctx.hybrid_sort_fallbacks() - fallbacks0
    per_step = [a.elapsed_time(b) for a, b in ev]
    t = sum(per_step) / 1e3
    kinds = [ctx.hybrid_profile_read(k) for k in range(9)]
    ctx.hybrid_profile(False)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_max = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    far_s = kinds[0][0] / 1e3 / max(kinds[0][1], 1)
    achieved = FLOPS_PER_INTERACTION * inter_far / steps / far_s / 1e12
    out = s.numpy()
    a_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)
    a_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)
    ferr = force_error_rms(out, a_s, a_h, eps, nsample=256)
    names = ["far_pair", "near_pair", "walk", "tree_build", "kick_drift", "sort", "topology", "moments", "groups"]
    ms = {nm: kinds[k][0] / steps for k, nm in enumerate(names)}
    ctx.close()
    del s, out, a_s, a_h
    torch.cuda.empty_cache()
    cpu = c3_cpu_leg(st, P) if with_cpu else None
    return {
        "workload": C3_NAME % n, "N": n, "metric": METRIC, "value": n * steps / t, "unit": METRIC, "steps": steps,
        "warmup": warmup, "ms_per_step": 1e3 * t / steps, "ms_median": sorted(per_step)[len(per_step) // 2],
        "ms_max": max(per_step), "dtype": "f32", "l2": "inputs larger than L2", "ic_seconds": t_ic,
        "autotuned": {"n_crit": chosen[0], "threads_per_group": chosen[1], "tile_depth": chosen[2]},
        "nodes": nodes, "groups": groups,
        "interactions_per_s": (inter_far + P.n_hard * inter_near) / t,
        "soft_interactions_per_step": (inter_far + inter_near) / steps,
        "hard_interactions_per_substep": inter_near / steps,
        "force_err_rms_vs_direct": ferr,
        "kernel_ms_per_step": ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_pair_f32 far (cells + far particles, soft force)",
                     "peak_note": "FP32 CUDA-core peak: %d SMs x 128 lanes x 2 flop x %.0f MHz (max SM clock)" %
                                  (props.multi_processor_count, sm_max)},
        "hbm_stages": hbm_stages(n, P.n_hard, ms, nodes),
        "gpu_launches": launches, "sort_fallbacks": fallbacks, "clocks": clk, "cpu_baseline": cpu,
    }


def run_c3(args):
    from paper_1406_6158_gb300 import build as cuda_build
    cuda_build.build()
    r = c3_record(args, args.steps, args.warmup, with_cpu=not args.no_cpu_baseline)
    line = {
        "metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": 1, "steps": r["steps"],
        "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "N": r["N"], "l2": r["l2"], "ic_seconds": r["ic_seconds"],
                   "autotuned": r["autotuned"]},
    }
    line.update({k: r[k] for k in ("interactions_per_s", "soft_interactions_per_step", "hard_interactions_per_substep",
                                   "force_err_rms_vs_direct", "kernel_ms_per_step", "roofline", "hbm_stages",
                                   "gpu_launches", "sort_fallbacks", "clocks", "cpu_baseline", "ms_median", "ms_max",
                                   "nodes", "groups")})
    print(json.dumps(line), flush=True)
    return 0


def paper_params(n):
    """The paper's parameter set for the Plummer model (Sec. IV-A): eps = 0.1 N^-0.26, dt_h = eps / sigma_v with
    sigma_v = 0.65, n = 4 hard steps per soft step, R1 = 1.03 N^-1/3, R2 = 2 R1, absolute MAC with a_err = 2^-8."""
    eps = 0.1 * n ** -0.26
    R1 = 1.03 * n ** (-1.0 / 3.0)
    return dict(eps=eps, dt_h=eps / 0.65, R1=R1, R2=2 * R1, a_err=2.0 ** -8, n_hard=4)


def run_paper(args):
    """Hybrid against normal tree on one GPU with the paper's parameters (Sec. IV-B, IV-D, Eq. 16).

    Three contexts on the same Plummer sphere, each autotuned, FP32 pairs on FP64 state:
      hybrid  n = 4 (one soft step and three hard steps per dt_s = 4 dt_h)      -> T_hybrid per dt_s
      soft    n = 1, dt_s = dt_h (the soft step alone)                          -> T_soft
      normal  R1 = R2 = 0 (K = 0: one tree force per step), dt_n = dt_h         -> T_tree per step
    T_hard = (T_hybrid - T_soft) / (n - 1); R_hybrid = T_hybrid / (n T_tree), which is Eq. 16's
    ((n-1) T_hard + T_soft) / (n T_tree) with the measured times (no domain decomposition on one GPU).
    The hard force alone (walk + near pairs of a hard step) is compared with the normal tree's force (walk +
    pairs) from a separate pass with every stage bracketed. Energy drift of the hybrid and the normal run over
    the same simulated time (dt_h = dt_n, as the paper sets them), for N <= ENERGY_MAX_N."""
    import numpy as np
    import torch
    from paper_1406_6158_gb300 import build as cuda_build
    from paper_1406_6158_gb300 import hybrid, ics
    cuda_build.build()
    sizes = [args.n] if args.n != N_DEFAULT else [1 << 18, 1 << 20, 1 << 22]
    stream = torch.cuda.Stream()           # a stream of its own: the library replays captured CUDA graphs on it
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    K = max(4, min(args.steps, 32))
    rows, clocks = [], ClockSampler(0)
    clocks.start()
    for n in sizes:
        pp = paper_params(n)
        st = ics.plummer(n, 4)
        forms = {
            "hybrid": dict(R1=pp["R1"], R2=pp["R2"], n_hard=pp["n_hard"], dt_soft=pp["n_hard"] * pp["dt_h"], k=K),
            "soft": dict(R1=pp["R1"], R2=pp["R2"], n_hard=1, dt_soft=pp["dt_h"], k=K),
            "normal": dict(R1=0.0, R2=0.0, n_hard=1, dt_soft=pp["dt_h"], k=pp["n_hard"] * K),
        }
        res = {}
        for name, f in forms.items():
            P = hybrid.Params(eps=pp["eps"], R1=f["R1"], R2=f["R2"], dt_soft=f["dt_soft"], n_hard=f["n_hard"],
                              a_err=pp["a_err"], mac=1, n_leaf=16, n_crit=64, precision=1)
            ctx = hybrid.Context(P, stream)
            s = hybrid.System(st, precision=1, ids=False)
            chosen, _ = ctx.hybrid_autotune(s)
            ctx.hybrid_step(s, 0)
            # direct FP64 summation on the device is O(N^2) on GB300's FP64 pipe: small systems only
            with_energy = name != "soft" and n <= ENERGY_MAX_N
            e0 = sum(ctx.hybrid_energy(s)) if with_energy else None
            for _ in range(3):
                ctx.hybrid_step(s, 1)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(f["k"])]
            torch.cuda.synchronize()
            for k in range(f["k"]):
                flush.zero_()
                ev[k][0].record(stream)
                ctx.hybrid_step(s, 1)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            t = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / f["k"]
            e1 = sum(ctx.hybrid_energy(s)) if with_energy else None
            kp = min(f["k"], 16)
            ctx.hybrid_profile(2)
            ctx.hybrid_profile_read(0, reset=True)
            for _ in range(kp):
                ctx.hybrid_step(s, 1)
            torch.cuda.synchronize()
            kinds = [ctx.hybrid_profile_read(k)[0] / kp / 1e3 for k in range(5)]   # far, near, walk, tree, kick
            ctx.hybrid_profile(0)
            res[name] = dict(t=t, force=kinds[0] + kinds[1] + kinds[2], tree=kinds[3],
                             drift=abs(e1 - e0) / abs(e0) if with_energy else None, steps=3 + f["k"], tuned=list(chosen))
            if name == "hybrid":
                out = s.numpy()
                a_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)
                a_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)
                res[name]["ferr"] = force_error_rms(out, a_s, a_h, pp["eps"], nsample=256)
            ctx.close()
        nh = pp["n_hard"]
        T_hyb, T_soft, T_tree = res["hybrid"]["t"], res["soft"]["t"], res["normal"]["t"]
        T_hard = (T_hyb - T_soft) / (nh - 1)
        hard_force = (res["hybrid"]["force"] - res["soft"]["force"]) / (nh - 1)
        rows.append({
            "N": n, "eps": pp["eps"], "dt_h": pp["dt_h"], "R1": pp["R1"], "R2": pp["R2"],
            "ms": {"T_hybrid_per_dt_s": 1e3 * T_hyb, "T_soft": 1e3 * T_soft, "T_hard": 1e3 * T_hard,
                   "T_tree": 1e3 * T_tree, "hard_force": 1e3 * hard_force, "normal_force": 1e3 * res["normal"]["force"]},
            "T_hard_over_T_soft": T_hard / T_soft,
            "T_hard_over_T_tree": T_hard / T_tree,
            "T_soft_over_T_tree": T_soft / T_tree,
            "hard_force_over_normal_force": hard_force / res["normal"]["force"],
            "R_hybrid": T_hyb / (nh * T_tree),
            "energy_drift": {"hybrid": res["hybrid"]["drift"], "normal": res["normal"]["drift"],
                             "hybrid_soft_steps": res["hybrid"]["steps"], "normal_steps": res["normal"]["steps"]},
            "force_err_rms_vs_direct": res["hybrid"]["ferr"],
            "particle_steps_per_s": {"hybrid": n / T_hyb, "normal": n / (nh * T_tree)},
            "autotuned": {k: v["tuned"] for k, v in res.items()},
        })
    clk = clocks.stop()
    head = rows[len(rows) // 2]
    line = {
        "metric": METRIC, "value": head["particle_steps_per_s"]["hybrid"], "unit": METRIC, "n_gpus": 1,
        "steps": K, "warmup": 3, "ms_per_step": head["ms"]["T_hybrid_per_dt_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "Plummer sphere seed 4 with the paper's parameters: eps=0.1N^-0.26, dt_h=eps/0.65, "
                               "n=4, R1=1.03N^-1/3, R2=2R1, absolute MAC a_err=2^-8; FP32 pairs, FP64 state; "
                               "value at N=%d" % head["N"],
                   "l2": "flushed (256 MiB write) before every timed step"},
        "paper_comparison": rows,
        "paper_values": {"T_hard_over_T_soft": "about 0.6 (Sec. IV-C, 32M particles, many GPUs)",
                         "hard_force_over_normal_force": "about 0.4 (Sec. IV-B, N 256k-4096k)",
                         "R_hybrid": "0.8-0.9 measured, 0.7 from Eq. 16 with its assumptions (Sec. IV-D)"},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-reuse", action="store_true", help="skip the reused-neighbour-list measurement")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the compact large and batched records of the default run")
    ap.add_argument("--ref-max-seconds", type=float, default=120.0,
                    help="time box of the reference arm's timed steps (the oracle on the host cores)")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per soft-pair launch from an ncu capture of this workload")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "served", "large", "paper"],
                    help="single: one Plummer sphere (default); batched: the 512-system ensemble; "
                         "served: the Poisson request stream; large: the 2^24 Hernquist sphere; "
                         "paper: hybrid against normal tree with the paper's parameters")
    ap.add_argument("--tune", default="auto",
                    help="auto (autotuner) or n_crit,threads_per_group,tile_depth for the single and large workloads")
    ap.add_argument("--c4-count", type=int, default=512)
    ap.add_argument("--c5-count", type=int, default=100)
    ap.add_argument("--c5-max-seconds", type=float, default=600.0)
    ap.add_argument("--verbose", action="store_true")
    args = ap.parse_args()
    w = workload(args.n)
    if args.workload == "batched" and args.impl == "gb300":
        args.warmup = max(args.warmup, 3)
        return run_c4(args)
    if args.workload == "served" and args.impl == "gb300":
        return run_c5(args)
    if args.workload == "large" and args.impl == "gb300":
        return run_c3(args)
    if args.workload == "paper" and args.impl == "gb300":
        return run_paper(args)
    if args.impl == "reference":
        return run_reference(args, w)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch
    from paper_1406_6158_gb300 import build as cuda_build
    from paper_1406_6158_gb300 import hybrid, ics

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(hybrid.LIB_PATH):
        cuda_build.build()
    if dist:
        dist.barrier()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    P = hybrid.Params(eps=w["eps"], theta=w["theta"], R1=w["R1"], R2=w["R2"], dt_soft=w["dt_soft"],
                      n_hard=w["n_hard"], n_leaf=w["n_leaf"], n_crit=w["n_crit"], precision=1)
    stream = torch.cuda.Stream()           # a stream of its own: the library replays captured CUDA graphs on it
    torch.cuda.set_stream(stream)
    ctx = hybrid.Context(P, stream)
    st = ics.plummer(w["n"], w["seed"])
    s = hybrid.System(st, precision=1)
    if args.tune == "auto":
        chosen, _ = ctx.hybrid_autotune(s)     # n_crit, threads per group, staging depth (untimed)
    else:                                      # a fixed choice, e.g. to profile the autotuned configuration
        chosen = tuple(int(v) for v in args.tune.split(","))
        ctx.hybrid_autotune(s, [chosen])
    ctx.hybrid_step(s, 0)                      # forces at the initial positions
    e_start = sum(ctx.hybrid_energy(s))        # softened total energy by direct FP64 summation (device)
    for _ in range(args.warmup):
        ctx.hybrid_step(s, 1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # ---- device-timed region: inputs resident in HBM, L2 flushed before every step ----
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.hybrid_profile(1)                      # the pair kernels only: two event nodes per launch
    for k in range(9):
        ctx.hybrid_profile_read(k, reset=True)
    launches0 = ctx.hybrid_launch_count()
    fallbacks0 = ctx.hybrid_sort_fallbacks()
    inter_far = inter_near = 0
    barrier()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.hybrid_step(s, 1)
        ev[k][1].record(stream)
        fi, ni = ctx.hybrid_interactions()     # pairs of the far and near kernels of the step's soft evaluation
        inter_far += fi
        inter_near += ni
    barrier()
    clk = clocks.stop()
    launches = ctx.hybrid_launch_count() - launches0
    fallbacks = ctx.hybrid_sort_fallbacks() - fallbacks0
    per_step = [a.elapsed_time(b) for a, b in ev]
    t_steps = sum(per_step) / 1e3
    nodes, groups = ctx.tree_info()            # the tree of the last timed build
    soft_ms, soft_n = ctx.hybrid_profile_read(0)
    hard_ms, hard_n = ctx.hybrid_profile_read(1)
    ctx.hybrid_profile_read(0, reset=True)     # a reset clears every kind
    # stage breakdown from a separate profiled pass (every stage bracketed: the brackets cost time)
    kp = min(args.steps, 50)
    ctx.hybrid_profile(2)
    for _ in range(kp):
        ctx.hybrid_step(s, 1)
    torch.cuda.synchronize()
    stage = [ctx.hybrid_profile_read(k)[0] / kp for k in range(9)]
    ctx.hybrid_profile_read(0, reset=True)
    ctx.hybrid_profile(0)
    value, t_steps = job_rate(w["n"] * args.steps, t_steps, dist)
    e_end = sum(ctx.hybrid_energy(s))
    energy = {"rel_drift": abs(e_end - e_start) / abs(e_start), "E_start": e_start, "E_end": e_end,
              "soft_steps": args.warmup + args.steps + kp, "time": (args.warmup + args.steps + kp) * w["dt_soft"]}

    # ---- reused neighbour lists (skin > 0, an option outside the paper's scheme), same workload ----
    reuse = None
    if not args.no_reuse:
        P2 = hybrid.Params(eps=w["eps"], theta=w["theta"], R1=w["R1"], R2=w["R2"], dt_soft=w["dt_soft"],
                           n_hard=w["n_hard"], n_leaf=w["n_leaf"], n_crit=w["n_crit"], precision=1, skin=REUSE_SKIN)
        ctx2 = hybrid.Context(P2, stream)
        s2 = hybrid.System(st, precision=1)
        ctx2.hybrid_autotune(s2, [tuple(chosen)])
        ctx2.hybrid_step(s2, 0)
        r_e0 = sum(ctx2.hybrid_energy(s2))
        for _ in range(args.warmup):
            ctx2.hybrid_step(s2, 1)
        kr = max(3, args.steps // 3)
        evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kr)]
        l0 = ctx2.hybrid_launch_count()
        clocks2 = ClockSampler(local)
        barrier()
        clocks2.start()
        for k in range(kr):
            flush.zero_()
            evr[k][0].record(stream)
            ctx2.hybrid_step(s2, 1)
            evr[k][1].record(stream)
        barrier()
        clk2 = clocks2.stop()
        per = [a.elapsed_time(b) for a, b in evr]
        tr = sum(per) / 1e3
        r_e1 = sum(ctx2.hybrid_energy(s2))
        rv, tr = job_rate(w["n"] * kr, tr, dist)
        reuse = {"skin": REUSE_SKIN, "value": rv, "unit": METRIC, "ms_per_step": 1e3 * tr / kr, "steps": kr,
                 "gpu_launches_per_step": (ctx2.hybrid_launch_count() - l0) / kr,
                 "ms_median": sorted(per)[len(per) // 2], "ms_max": max(per), "clocks": clk2,
                 "energy_rel_drift": abs(r_e1 - r_e0) / abs(r_e0), "energy_soft_steps": 1 + args.warmup + kr,
                 "note": "hard steps 1..n-1 reuse the tree and neighbour lists of the last build (lists to R2 + "
                         "skin); not the paper's scheme, which rebuilds every hard step"}
        ctx2.close()

    # ---- end to end through the C-ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        keys = ["x", "y", "z", "vx", "vy", "vz", "m", "ax_s", "ay_s", "az_s", "ax_h", "ay_h", "az_h", "id"]
        host = {k: s.t[k].detach().cpu().pin_memory() for k in keys}
        h2d = sum(host[k].numel() * host[k].element_size() for k in keys)
        ke = max(3, args.steps // 2)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            for k in keys:
                s.t[k].copy_(host[k], non_blocking=True)
            ctx.hybrid_step(s, 1)
            for k in keys:
                host[k].copy_(s.t[k], non_blocking=True)
            torch.cuda.current_stream().synchronize()
        e1.record(stream)
        barrier()
        te = e0.elapsed_time(e1) / 1e3
        e2e_value, te = job_rate(w["n"] * ke, te, dist)
        e2e = {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
               "steps": ke}

    out = s.numpy()
    a_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)
    a_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)

    # ---- roofline of the dominant kernel (soft pair, FP32 CUDA-core bound) ----
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    soft_avg_s = (soft_ms / 1e3) / max(soft_n, 1)
    per_launch_flops = FLOPS_PER_INTERACTION * inter_far / max(args.steps, 1)
    achieved = per_launch_flops / soft_avg_s / 1e12 if soft_avg_s > 0 else None
    traffic = args.traffic_bytes if args.traffic_bytes is not None else FAR_TRAFFIC_BYTES.get(tuple(chosen))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum of one far launch of this "
                                   "variant on this workload, from an ncu capture of the current kernel (mean "
                                   "of two launches); not measured in this run") if traffic else
                                  "no capture of the chosen variant",
                "kernel": "k_pair_f32 far (cells + far particles, soft force)",
                "peak_note": "FP32 CUDA-core peak: %d SMs x 128 lanes x 2 flop x %.0f MHz (max SM clock)" %
                             (props.multi_processor_count, sm_max)}

    ctx.close()

    # ---- compact records of the large and the batched workloads (one GPU) ----
    subs = {}
    if ws == 1 and not args.no_sub:
        import gc
        del s
        gc.collect()
        torch.cuda.empty_cache()
        large_steps = max(2, min(args.steps, 4))
        subs["large"] = c3_record(args, large_steps, 2, with_cpu=not args.no_cpu_baseline)
        gc.collect()
        torch.cuda.empty_cache()
        subs["batched"] = c4_record(args, max(3, min(args.steps, 5)), 3)
        torch.cuda.set_stream(stream)

    line = None
    if rank == 0:
        ferr = force_error_rms(out, a_s, a_h, w["eps"])
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            cpu = cpu_baseline(w)
        step_ms = 1e3 * t_steps / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "ms_median": sorted(per_step)[len(per_step) // 2],
            "ms_max": max(per_step), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(w), "N": w["n"], "parallelism": "replicas x%d" % ws,
                       "l2": "flushed (256 MiB write) before every timed step", "state": "f64",
                       "autotuned": {"n_crit": chosen[0], "threads_per_group": chosen[1],
                                     "tile_depth": chosen[2]}},
            # soft force: far + near pairs once per step; hard force: near pairs at each of the n_hard sub-steps
            "interactions_per_s": ws * (inter_far + w["n_hard"] * inter_near) / t_steps,
            "soft_interactions_per_step": (inter_far + inter_near) / args.steps,
            "hard_interactions_per_substep": inter_near / args.steps,
            "force_err_rms_vs_direct": ferr,
            "energy": energy,
            "kernel_ms_per_step": {"far_pair": soft_ms / args.steps, "near_pair": hard_ms / args.steps,
                                   "walk": stage[2], "tree_build": stage[3], "kick_drift": stage[4],
                                   "tree_parts": {"sort": stage[5], "topology": stage[6], "moments": stage[7],
                                                  "groups": stage[8]},
                                   "note": "far and near pair: the timed region; the other stages: a separate "
                                           "pass of %d steps with every stage bracketed; topology and groups "
                                           "run beside the permutation and the moments" % kp},
            "roofline": roofline,
            "reused_lists": reuse,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "sort_fallbacks": fallbacks,
            "clocks": clk,
            "tree": {"nodes": nodes, "groups": groups},
            "hbm_stages": hbm_stages(w["n"], w["n_hard"], {"sort": stage[5], "topology": stage[6],
                                                           "moments": stage[7], "kick_drift": stage[4]}, nodes),
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
