#!/usr/bin/env python3
"""Benchmark of the signed-particle WBRW hot path on GB300.

One bench step is one resampling period of the workload: regenerate the
particles from the histogram (Alg. 3), stream and branch them through
`resample_every` intervals (Alg. 1), and resample (sp1 annihilation or the sp2
signed bootstrap).  The default workload is the 2D Gaussian barrier at scale:
1e8 particles, FP32 state, 1200 x 512 cells, dt = 0.05, resampling every 10
intervals; 10 warm-up + 30 timed periods cover its 400 intervals.

metric: signed-particle steps per second including annihilation, i.e. the sum
over intervals of the particles alive at the start of the interval, divided
by the device time of all flight and resampling work.

`--impl reference` times the plain FP64 CPU oracle on the host instead,
on a bounded sample of the same workload.
Multi-GPU (`torchrun`): independent replicas, one per GPU, different seeds.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "signed-particle steps/s incl. annihilation (2D, 4D); batched+grad vs plain"
UNIT = "particle-steps/s"
L2_FLUSH_BYTES = 512 << 20      # > 129 MB of L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--strategy", default="sp1", choices=["sp1", "sp2", "wp"])
    ap.add_argument("--workload", default="gauss2d_fp32_n1e8",
                    choices=["gauss2d_fp32_n1e8", "gauss2d_fp64_n2e5", "batch2d_fp32_256",
                             "he4d_fp32_n5e7", "grad2d_fp32_64", "tdv2d_fp32_n1e8"])
    ap.add_argument("--group", type=int, default=4,
                    help="differentiation workload: parameter points per batch")
    ap.add_argument("--n-scale", type=float, default=1.0,
                    help="batched workload: scale every instance's particle count")
    ap.add_argument("--no-plain", action="store_true",
                    help="batched workload: skip the plain per-instance comparison")
    ap.add_argument("--particles", type=float, default=0,
                    help="override the particle count (profiling small cases)")
    ap.add_argument("--capacity-factor", type=float, default=4.0,
                    help="particle capacity as a multiple of the particle count")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every period kernel by kernel instead of replaying a CUDA graph")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape instead of autotuning it after warm-up")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(args):
    if args.workload == "grad2d_fp32_64":
        return workloads.scaled(workloads.GRAD_2D_FP32_64)
    if args.workload == "tdv2d_fp32_n1e8":
        wl = workloads.scaled(workloads.TDV_2D_FP32_1E8, strategy=args.strategy)
        if args.particles:
            wl["n_alpha"] = int(args.particles)
        return wl
    if args.workload == "batch2d_fp32_256":
        return workloads.scaled(workloads.BATCH_2D_FP32_256)
    if args.workload == "he4d_fp32_n5e7":
        wl = workloads.scaled(workloads.HE_4D_FP32_5E7)
        if args.particles:
            wl["n_alpha"] = int(args.particles)
        return wl
    base = (workloads.GAUSS_2D_FP32_1E8 if args.workload == "gauss2d_fp32_n1e8"
            else workloads.GAUSS_2D_FP64_2E5)
    wl = workloads.scaled(base, strategy=args.strategy)
    if args.particles:
        wl["n_alpha"] = int(args.particles)
    return wl


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), "wbrw_clocks_%d_%d.csv" % (gpu_index,
                                                                               os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on the host: CPU baseline and the reference arm
# ---------------------------------------------------------------------------
def oracle_period_rate(wl, n_sample, budget_s, max_periods=None):
    """Time the FP64 oracle, as it stands, on a sample of the workload:
    n_sample initial particles, full periods until budget_s has elapsed."""
    import oracle
    oracle.build()
    if wl.get("dim", 2) == 4:
        o = oracle.Oracle4(hbar=wl["hbar"], mass=wl["mass"], dt=wl["dt"], Z=wl["Z"], a=wl["a"],
                           xc=wl["xc"], lam=wl["lam"], nx=wl["nx"], nk=wl["nk"],
                           xmin=wl["xmin"], xmax=wl["xmax"], kmin=wl["kmin"], kmax=wl["kmax"],
                           ny=wl["ny"], nkap=wl["nkap"], n_alpha=n_sample, seed=wl["seed"])
    else:
        o = oracle.Oracle(hbar=wl["hbar"], mass=wl["mass"], dt=wl["dt"], gamma0=wl["gamma0"],
                          H=wl["H"], w=wl["w"], xc=wl["xc"], nx=wl["nx"], nk=wl["nk"],
                          xmin=wl["xmin"], xmax=wl["xmax"], kmin=wl["kmin"], kmax=wl["kmax"],
                          strategy=oracle.SP1 if wl["strategy"] == "sp1" else oracle.SP2,
                          n_alpha=n_sample, seed=wl["seed"], comps=tuple(wl.get("comps", ())))
    o.init_gauss(n_sample, wl["x0"], wl["sigma_x"], wl["k0"])
    times, psteps = [], []
    t_all = time.perf_counter()
    while True:
        p0 = o.ledger()["particle_steps"]
        t0 = time.perf_counter()
        o.step(wl["resample_every"])
        o.annihilate()
        times.append(time.perf_counter() - t0)
        psteps.append(o.ledger()["particle_steps"] - p0)
        if time.perf_counter() - t_all > budget_s or (max_periods and len(times) >= max_periods):
            break
    return times, psteps


def reference_arm(args, wl):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    n_sample = 200_000
    times, psteps = oracle_period_rate(wl, n_sample, budget_s=1e9,
                                       max_periods=args.warmup + args.steps)
    t = sum(times[args.warmup:])
    ps = sum(psteps[args.warmup:])
    value = ps / t if t > 0 else 0.0
    sample = ("%d-particle sample (of %d) of the same workload, %d-interval periods "
              "incl. annihilation, FP64 oracle, single thread"
              % (n_sample, int(wl["n_alpha"]), wl["resample_every"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(wl, args):
    d4 = wl.get("dim", 2) == 4
    pot = ("soft-Coulomb Z=%g a=%g ee=%g, tables %dx%d" % (wl["Z"], wl["a"], wl["lam"], wl["ny"],
                                                          wl["nkap"])
           if d4 else "gaussian H=%g w=%g" % (wl["H"], wl["w"]))
    if wl.get("comps"):
        pot = "time-dependent: " + " + ".join(
            "(%g%+g cos(%g t%+.4g)) gauss(w=%g, xc=%g)" % (c["a"], c["b"], c["om"], c["ph"], c["w"],
                                                         c["xc"]) for c in wl["comps"])
    return {"workload": wl["name"], "dim": 4 if d4 else 2, "particles": int(wl["n_alpha"]),
            "grid": [wl["nx"]] * (2 if d4 else 1) + [wl["nk"]] * (2 if d4 else 1),
            "dt": wl["dt"],
            "intervals_per_step": wl["resample_every"], "strategy": wl["strategy"],
            "precision": wl["precision"], "potential": pot,
            "l2": "flushed (512 MiB write) between timed steps",
            "cuda_graphs": not args.no_graph and wl["strategy"] == "sp1",
            "parallelism": "replicas x%d" % args.gpus}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def ours(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1709_02121_gb300 import build
    build.build()
    from paper_1709_02121_gb300 import Simulation, Simulation4, wbrw

    wl = workloads.scaled(wl, seed=wl["seed"] + rank)
    n = int(wl["n_alpha"])
    cap = int(args.capacity_factor * n) + (1 << 20)
    model = Simulation4 if wl.get("dim", 2) == 4 else Simulation
    sim = model(wl, capacity=cap, stream=torch.cuda.Stream())
    stream = sim.stream
    graphs = not args.no_graph and wl["strategy"] == "sp1"
    if graphs:
        sim.graph(True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    P = wl["resample_every"]
    tuning = warm_up(sim, args, P)
    barrier()

    c0 = sim.counters()
    wbrw.wbrw_profile(sim.ctx, True)  # clears what the last warm-up period recorded
    clocks = Clocks(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i)  # evict the histogram and plan from L2
        stream.wait_stream(torch.cuda.current_stream())  # the flush ends before the timing starts
        starts[i].record(stream)
        sim.run(P)
        ends[i].record(stream)
    barrier()
    clk = clocks.stop()
    kern_ms, kern_n = wbrw.wbrw_profile_read(sim.ctx)
    ev_ms, ev_n = wbrw.wbrw_profile_read_events(sim.ctx)
    c1 = sim.counters()
    t_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    psteps = c1["particle_steps"] - c0["particle_steps"]
    psteps_first = c1["particle_steps_first"] - c0["particle_steps_first"]
    launches = c1["launches"] - c0["launches"]

    # ---- end to end: host checkpoint in, one period, checkpoint + observables out
    e2e = None
    if not args.no_e2e:
        grid_h = torch.empty(sim.grid_counts().shape, dtype=torch.int32).pin_memory()
        g0, step0, epoch0 = sim.checkpoint(grid_h.numpy())
        e2e_steps = min(args.steps, 10)
        barrier()
        pe0 = sim.counters()["particle_steps"]
        t0 = time.perf_counter()
        T_last = None
        for i in range(e2e_steps):
            sim.restore(grid_h.numpy(), step0 if i == 0 else step, epoch0 if i == 0 else epoch)
            sim.run(P)
            _, step, epoch = sim.checkpoint(grid_h.numpy())
            _, _, T_last, _ = wbrw.wbrw_density(sim.ctx, wl["nx"], wl["nk"])
        te = time.perf_counter() - t0
        pe = sim.counters()["particle_steps"] - pe0
        e2e = {"value": pe / te, "unit": UNIT,
               "h2d_bytes_per_step": int(sim.cells * 4),
               "d2h_bytes_per_step": int(sim.cells * 4 + wl["nx"] * wl["nk"] * 8
                                         + wl["nx"] * 8 + 16),
               "steps": e2e_steps, "transmission_last": T_last}

    # ---- reduce over ranks: max time, summed particle-steps and e2e rate
    t_max, ps_all, e2e_sum = reduce_over_ranks(ws, t_ms, psteps, e2e["value"] if e2e else 0.0,
                                               "cuda")
    if e2e is not None:
        e2e["value"] = e2e_sum

    if rank == 0:
        value = ps_all / (t_max / 1e3)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        roof, roof2 = dominant(
            roofline(wl, kern_ms, kern_n, psteps_first, peaks, clk),
            roofline_event(wl, ev_ms, ev_n, c1["candidates"] - c0["candidates"],
                           c1["first_pairs"] - c0["first_pairs"], peaks, clk))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if wl["precision"] == "fp32" else "f64",
                "data": "synthetic", "config": config_of(wl, args),
                "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "roofline_secondary": roof2, "clocks": clk, "tuning": tuning,
                "live_particles_end": c1["live"],
                "particle_steps": psteps}
        if not args.no_cpu_baseline and ws == 1:
            times, pst = oracle_period_rate(wl, 1_000_000 if n >= 1_000_000 else n, budget_s=15.0)
            line["cpu_baseline"] = {
                "value": sum(pst) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d of the %d particles, %d full %d-interval periods incl. "
                          "annihilation, FP64 oracle, single thread"
                          % (min(n, 1_000_000), n, len(times), P)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    sim.close()


def ours_batch(args, spec):
    """The batched workload: all instances in one context and the same
    launches, timed like the plain workload; then the plain per-instance path
    (one context per instance, run one after the other on the same GPU) for
    the same periods, for comparison."""
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1709_02121_gb300 import build
    build.build()
    from paper_1709_02121_gb300 import Batch, Simulation, wbrw

    wl = workloads.scaled(spec, seed=spec["seed"] + rank)
    insts = workloads.batch_instances(wl, args.n_scale)
    n_total = sum(v["n_init"] for v in insts)
    cap = int(args.capacity_factor * n_total) + (1 << 20)
    sim = Batch(wl, insts, capacity=cap, stream=torch.cuda.Stream())
    stream = sim.stream
    graphs = not args.no_graph
    if graphs:
        sim.graph(True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    P = wl["resample_every"]
    tuning = warm_up(sim, args, P)
    barrier()
    c0 = sim.counters()
    wbrw.wbrw_profile(sim.ctx, True)  # clears what the last warm-up period recorded
    clocks = Clocks(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i)
        stream.wait_stream(torch.cuda.current_stream())  # the flush ends before the timing starts
        starts[i].record(stream)
        sim.run(P)
        ends[i].record(stream)
    barrier()
    clk = clocks.stop()
    kern_ms, kern_n = wbrw.wbrw_profile_read(sim.ctx)
    ev_ms, ev_n = wbrw.wbrw_profile_read_events(sim.ctx)
    c1 = sim.counters()
    t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    psteps = c1["particle_steps"] - c0["particle_steps"]
    psteps_first = c1["particle_steps_first"] - c0["particle_steps_first"]
    launches = c1["launches"] - c0["launches"]
    T_batch = sim.transmissions()

    # ---- end to end: every period resumes from the host checkpoint of all
    # instances and returns it, with the transmissions of every instance
    e2e = None
    if not args.no_e2e:
        m = len(insts)
        grid_h = torch.empty((m, wl["nx"], wl["nk"]), dtype=torch.int32).pin_memory()
        _, step, epoch = sim.checkpoint(grid_h.numpy())
        e2e_steps = min(args.steps, 5)
        barrier()
        pe0 = sim.counters()["particle_steps"]
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            sim.restore(grid_h.numpy(), step, epoch)
            sim.run(P)
            _, step, epoch = sim.checkpoint(grid_h.numpy())
            T_last = sim.transmissions()
        te = time.perf_counter() - t0
        pe = sim.counters()["particle_steps"] - pe0
        e2e = {"value": pe / te, "unit": UNIT,
               "h2d_bytes_per_step": int(m * wl["nx"] * wl["nk"] * 4),
               "d2h_bytes_per_step": int(m * wl["nx"] * wl["nk"] * 4 + m * 8),
               "steps": e2e_steps, "transmission_mean_last": float(np.mean(T_last))}
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # ---- the plain per-instance path: one context per instance on shared
    # buffers sized for the largest instance, the same warm-up and timed
    # periods, device time summed over the instances' timed periods
    plain = None
    if not args.no_plain:
        nmax = max(v["n_init"] for v in insts)
        base = workloads.scaled(wl, n_alpha=nmax)
        host = Simulation.__new__(Simulation)
        host.ninst = 1
        host._buffers(base, int(args.capacity_factor * nmax) + (1 << 20), 0, torch.cuda.Stream())
        t_plain, ps_plain = 0.0, 0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for v in insts:
            cfg = wbrw.Config(2, host.cfg.precision, host.cfg.strategy, wl["hbar"], wl["mass"],
                              wl["dt"], 0.0, wl["nx"], wl["nk"], wl["xmin"], wl["xmax"],
                              wl["kmin"], wl["kmax"], P, int(v["n_alpha"]), int(wl["seed"]))
            pot = wbrw.Potential(wbrw.POT_GAUSSIAN, v["H"], v["w"], v["xc"])
            ctx = wbrw.wbrw_init(cfg, pot, host.bufs, int(v["n_init"]), v["x0"], v["sigma_x"],
                                 v["k0"], host.stream.cuda_stream)
            if graphs:
                wbrw.wbrw_graph(ctx, True)
            for _ in range(args.warmup):
                wbrw.wbrw_run(ctx, P)
            p0 = wbrw.wbrw_counters(ctx)["particle_steps"]
            flush.fill_(0)
            host.stream.wait_stream(torch.cuda.current_stream())
            ev[0].record(host.stream)
            for _ in range(args.steps):
                wbrw.wbrw_run(ctx, P)
            ev[1].record(host.stream)
            torch.cuda.synchronize()
            t_plain += ev[0].elapsed_time(ev[1])
            ps_plain += wbrw.wbrw_counters(ctx)["particle_steps"] - p0
            wbrw.wbrw_destroy(ctx)
        plain = {"value": ps_plain / (t_plain / 1e3), "unit": UNIT,
                 "ms_per_step": t_plain / args.steps, "particle_steps": ps_plain,
                 "path": "one context per instance, instances one after the other",
                 "cuda_graphs": graphs}

    t_max, ps_all, e2e_sum = reduce_over_ranks(ws, t_ms, psteps, e2e["value"] if e2e else 0.0,
                                               "cuda")
    if e2e is not None:
        e2e["value"] = e2e_sum
    if rank == 0:
        value = ps_all / (t_max / 1e3)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        roof, roof2 = dominant(
            roofline(wl, kern_ms, kern_n, psteps_first, peaks, clk),
            roofline_event(wl, ev_ms, ev_n, c1["candidates"] - c0["candidates"],
                           c1["first_pairs"] - c0["first_pairs"], peaks, clk))
        ns = [v["n_init"] for v in insts]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": wl["name"], "instances": len(insts),
                           "particles": int(n_total), "particles_min_max": [min(ns), max(ns)],
                           "grid_per_instance": [wl["nx"], wl["nk"]], "dt": wl["dt"],
                           "intervals_per_step": P, "strategy": "sp1", "precision": "fp32",
                           "cuda_graphs": graphs,
                           "l2": "flushed (512 MiB write) between timed steps",
                           "parallelism": "replicas x%d" % ws},
                "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "roofline_secondary": roof2, "clocks": clk, "tuning": tuning,
                "live_particles_end": c1["live"], "particle_steps": psteps,
                "transmission_mean": float(np.mean(T_batch))}
        if plain is not None:
            plain["speedup_of_batch"] = plain["ms_per_step"] / (t_ms / args.steps)
            line["plain_per_instance"] = plain
        if not args.no_cpu_baseline and ws == 1:
            # the oracle on one instance of the batch (the first), sampled
            v = insts[0]
            one = workloads.scaled(wl, H=v["H"], w=v["w"], k0=v["k0"])
            n_s = min(v["n_init"], 200_000)
            times, pst = oracle_period_rate(one, n_s, budget_s=15.0)
            line["cpu_baseline"] = {
                "value": sum(pst) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "instance 0 (H=%.3g, w=%.3g, k0=%.3g), %d initial particles, %d "
                          "full %d-interval periods incl. annihilation, FP64 oracle, single "
                          "thread" % (v["H"], v["w"], v["k0"], n_s, len(times), P)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def warm_up(sim, args, P):
    """W untimed periods: W - 1, the launch-shape autotuning (which releases
    the period graphs), then profiling on and the last one, which captures
    the period graph again with the profiling events, so that no capture
    falls in the timed region.  Profiling stays on until the end (switching
    it captures the graphs again)."""
    from paper_1709_02121_gb300 import wbrw
    for _ in range(max(args.warmup - 1, 0)):
        sim.run(P)
    tuning = autotune(sim, args)
    wbrw.wbrw_profile(sim.ctx, True)
    sim.run(P)
    return tuning


def autotune(sim, args):
    """Pick the launch shape by timing one period under each (results do not
    depend on it); the run continues from where it was."""
    if args.no_autotune:
        b, p = sim.tuning()
        return {"blocks_per_sm": b, "event_passes": p, "autotuned": False}
    (b, p), table = sim.autotune(trials=2)
    return {"blocks_per_sm": b, "event_passes": p, "autotuned": True,
            "period_ms": [[round(float(v), 4) for v in row] for row in table]}


def ours_grad(args, spec):
    """The differentiation workload: T(H, w) and its likelihood-ratio
    derivatives for a batch of parameter points.  Times the forward batch
    (no tangents) and the gradient batch (tangent mode, the replay that
    autograd's backward runs) on the same points and periods, and reports
    the cost of the gradient against central finite differences, which need
    four forward runs per point for two parameters."""
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1709_02121_gb300 import build
    build.build()
    from paper_1709_02121_gb300 import Batch, wbrw

    wl = workloads.scaled(spec, seed=spec["seed"] + rank)
    pts = workloads.grad_points(wl)
    # a group spread over the parameter square (the sweep runs 64 / group
    # such batches one after another)
    idx = np.linspace(0, len(pts) - 1, args.group).round().astype(int)
    pts = [pts[i] for i in idx]
    n = max(1, int(round(wl["n_per_point"] * args.n_scale)))
    insts = [dict(H=h, w=v, xc=wl["xc"], x0=wl["x0"], sigma_x=wl["sigma_x"], k0=wl["k0"],
                  n_init=n, n_alpha=n) for h, v in pts]
    cap = int(args.capacity_factor * n * len(insts)) + (1 << 20)
    P = wl["resample_every"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def arm(tangent):
        b = Batch(dict(wl, tangent=tangent), insts, cap, stream=torch.cuda.Stream())
        stream = b.stream
        if not args.no_graph:
            b.graph(True)
        for _ in range(args.warmup):
            b.run(P)
        barrier()
        c0 = b.counters()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        clocks = Clocks(local)
        clocks.start()
        for i in range(args.steps):
            flush.fill_(i)
            stream.wait_stream(torch.cuda.current_stream())
            ev[2 * i].record(stream)
            b.run(P)
            ev[2 * i + 1].record(stream)
        barrier()
        clk = clocks.stop()
        c1 = b.counters()
        t_ms = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps))
        T = b.transmissions()
        g = b.transmission_gradients() if tangent else None
        res = {"t_ms": t_ms, "psteps": c1["particle_steps"] - c0["particle_steps"],
               "launches": c1["launches"] - c0["launches"], "live": c1["live"], "T": T,
               "grad": g, "clk": clk}
        b.close()
        del b
        torch.cuda.empty_cache()
        return res

    fwd = arm(False)
    bwd = arm(True)
    if not np.array_equal(fwd["T"], bwd["T"]):
        raise RuntimeError("the tangent run did not reproduce the forward run")
    t_max, ps_all, _ = reduce_over_ranks(ws, bwd["t_ms"], bwd["psteps"], 0.0, "cuda")
    if rank == 0:
        value = ps_all / (t_max / 1e3)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f32 tangent weights)",
                "data": "synthetic",
                "config": {"workload": wl["name"], "points_in_batch": len(insts),
                           "points": [[round(h, 4), round(v, 4)] for h, v in pts],
                           "particles_per_point": n, "grid": [wl["nx"], wl["nk"]],
                           "dt": wl["dt"], "intervals_per_step": P, "strategy": "sp1",
                           "precision": "fp32 state and tangent weights",
                           "cuda_graphs": not args.no_graph,
                           "l2": "flushed (512 MiB write) between timed steps",
                           "parallelism": "replicas x%d" % ws},
                "e2e": None, "gpu_launches": bwd["launches"], "clocks": bwd["clk"],
                "particle_steps": bwd["psteps"],
                "note": "value: the gradient run (tangent mode), whose particle-steps include "
                        "the sign-0 tangent particles",
                "forward": {"value": fwd["psteps"] / (fwd["t_ms"] / 1e3), "unit": UNIT,
                            "ms_per_step": fwd["t_ms"] / args.steps},
                "gradient_cost_vs_forward": bwd["t_ms"] / fwd["t_ms"],
                "lr_speedup_vs_central_differences": 4.0 * fwd["t_ms"] / bwd["t_ms"],
                "T": [round(float(x), 6) for x in bwd["T"]],
                "dT_dH": [round(float(x), 6) for x in bwd["grad"][:, 0]],
                "dT_dw": [round(float(x), 6) for x in bwd["grad"][:, 1]]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def reduce_over_ranks(ws, t_ms, psteps, e2e_value, device):
    """Whole-job numbers of the replicas: the slowest rank's time, and the
    particle-steps and end-to-end rates of all ranks summed."""
    if ws <= 1:
        return t_ms, psteps, e2e_value
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    sums = torch.tensor([float(psteps), float(e2e_value)], dtype=torch.float64, device=device)
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(sums[0].item()), float(sums[1].item())


def dominant(*roofs):
    """The rooflines ordered by the kernel's total time in the timed region:
    (the dominant kernel's, the other's)."""
    r = sorted((x for x in roofs if x), key=lambda x: -x["total_ms"])
    return (r[0] if r else None), (r[1] if len(r) > 1 else None)


def _int_peak(peaks, clk):
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
    return 152 * 64 * sm_mhz * 1e6 / 1e9, sm_mhz


def roofline_event(wl, ev_ms, ev_n, cand, pairs, peaks, clk):
    """Roofline of the event kernel (k_event), which performs the first event
    of every candidate interval: the kick, the acceptance and, for an
    accepted event, the pair; in FP32 the offspring then fly to the end of
    the period into the histogram inside the same kernel.  Its work is
    Philox calls, the entry decode and the histogram index arithmetic on the
    integer pipe, with a few transcendental functions per event.

    achieved = (INT_OPS_EVENT per candidate x candidates + per pair x
    first-event pairs) of the timed region / the kernel's summed CUDA-event
    time; both counts are device counters.
    peak = 152 SMs x 64 INT32 lanes x the median SM clock sampled during the
    timed region."""
    if not ev_n or ev_ms <= 0 or cand <= 0:
        return None
    key = wl["precision"] + ("_4d" if wl.get("dim", 2) == 4 else "")
    per_cand, per_pair = INT_OPS_EVENT[key]
    peak, sm_mhz = _int_peak(peaks, clk)
    ops = per_cand * cand + per_pair * pairs
    ach = ops / (ev_ms / 1e3) / 1e9
    tpc = TRAFFIC_PER_CANDIDATE.get(key)
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gop/s",
            "frac": ach / peak, "traffic": tpc and tpc * cand / ev_n,
            "kernel": "k_event<%s%s,bin>" % (wl["precision"],
                                             ",4d" if wl.get("dim", 2) == 4 else ""),
            "launch_ms": ev_ms / ev_n, "launches": ev_n, "total_ms": ev_ms,
            "candidates_per_launch": cand / ev_n, "first_pairs_per_candidate": pairs / cand,
            "int_ops_per_candidate": ops / cand,
            "peak_basis": "152 SM x 64 INT32 lanes x %.0f MHz (median SM clock sampled in the "
                          "timed region)" % sm_mhz}


def roofline(wl, kern_ms, kern_n, psteps_first, peaks, clk):
    """Roofline of the first wave: the fused regenerate + flight + histogram
    pass that carries the particles present at the start of each period.
    The particle state never leaves registers and HBM sees only the
    candidate queue, so the pass is bound by the integer pipe
    (Philox4x32-10 is 32-bit multiplies and XORs).

    achieved = the algorithm's integer operations per first-wave particle
    and period (INT_OPS_PER_PARTICLE, counted below) / the period's
    intervals x the first-wave particle-steps of one launch / the launch's
    average CUDA-event time.
    peak = 152 SMs x 64 INT32 lanes x the median SM clock sampled during the
    timed region (one integer operation per lane per cycle)."""
    if not kern_n or kern_ms <= 0:
        return None
    key = wl["precision"] + ("_4d" if wl.get("dim", 2) == 4 else "")
    R = wl["resample_every"]
    base, per_interval = INT_OPS_PER_PARTICLE[key]
    ops = (base + per_interval * R) / R
    per_launch_ms = kern_ms / kern_n
    peak, sm_mhz = _int_peak(peaks, clk)
    ach = ops * (psteps_first / kern_n) / (per_launch_ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gop/s",
            "frac": ach / peak, "traffic": TRAFFIC_PER_PSTEP.get(key) and
            TRAFFIC_PER_PSTEP[key] * psteps_first / kern_n,
            "kernel": "k_flight<%s%s,regen,bin>" % (wl["precision"],
                                                     ",4d" if wl.get("dim", 2) == 4 else ""),
            "launch_ms": per_launch_ms, "launches": kern_n, "total_ms": kern_ms,
            "first_wave_particle_steps_per_launch": psteps_first / kern_n,
            "int_ops_per_particle_step": ops,
            "peak_basis": "152 SM x 64 INT32 lanes x %.0f MHz (median SM clock sampled in the "
                          "timed region)" % sm_mhz}


# Integer operations per first-wave particle and period of R intervals
# (per particle, per interval).
# A Philox4x32-10 call counts 100 (10 rounds of two 32x32->64 multiplies as
# lo and hi, four XORs, two key additions).  FP32: one call per particle
# (regeneration offsets and the first candidate gap) plus the cell decode,
# in-cell coordinates, gap bits and histogram index.  FP64: the
# regeneration call(s) plus one call per interval for the candidate test.
INT_OPS_PER_PARTICLE = {"fp32": (120, 0), "fp32_4d": (135, 0),
                        "fp64": (116, 100), "fp64_4d": (230, 100)}
# DRAM bytes per first-wave particle-step measured by ncu (profiles/), or None
TRAFFIC_PER_PSTEP = {"fp32": 0.577, "fp64": None, "fp32_4d": 1.11, "fp64_4d": None}

# Integer operations of the event kernel (per candidate interval, per pair
# of its first event).  A candidate: the Philox calls of its first event (one
# in FP32 2D, where it also gives the life-length; the life-length call and
# the event's call in FP32 4D; one plus the event's two in FP64) and about 20
# for the entry decode, the uniforms and the next candidate interval, plus
# the guided table search of the 4D kick.  A pair: the Philox call of the
# offspring ids and, per offspring, about 20 for the first-event bits, the
# kill test, the cell index and the histogram index (30 with the four 4D
# indices).
INT_OPS_EVENT = {"fp32": (120, 140), "fp32_4d": (240, 160),
                 "fp64": (320, 140), "fp64_4d": (340, 160)}
# DRAM bytes per candidate interval of the event kernel measured by ncu
# (profiles/), or None
TRAFFIC_PER_CANDIDATE = {"fp32": 31.2, "fp64": None, "fp32_4d": 48.6, "fp64_4d": None}


def main():
    args = parse()
    wl = workload(args)
    if args.impl == "reference":
        reference_arm(args, wl)
    elif args.workload == "batch2d_fp32_256":
        ours_batch(args, wl)
    elif args.workload == "grad2d_fp32_64":
        ours_grad(args, wl)
    else:
        ours(args, wl)


if __name__ == "__main__":
    main()
