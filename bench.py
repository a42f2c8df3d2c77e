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

The default line also carries, under "secondary", the other parts of the
metric measured the same way on the same GPU: the 1e8 workload with the sp2
bootstrap, the 4D Helium-like workload, the batch of 256 instances against
the plain per-instance path, and the gradient of T(H, w) at 64 parameter
points against the forward run.

`--impl reference` times the plain FP64 CPU oracle on the host instead,
on a bounded sample of the same workload, on all host cores.
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


def parse(argv=None):
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
    ap.add_argument("--points", type=int, default=64,
                    help="differentiation workload: parameter points swept (of the 64)")
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
    ap.add_argument("--tuning", default="",
                    help="BLOCKS_PER_SM,EVENT_PASSES: this launch shape instead of autotuning")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: leave out the secondary workloads")
    return ap.parse_args(argv)


def workload(args):
    if args.workload == "grad2d_fp32_64":
        return workloads.scaled(workloads.GRAD_2D_FP32_64)
    if args.workload == "tdv2d_fp32_n1e8":
        wl = workloads.scaled(workloads.TDV_2D_FP32_1E8, strategy=args.strategy)
        if args.particles:
            wl["n_alpha"] = int(args.particles)
        return wl
    if args.workload == "batch2d_fp32_256":
        return workloads.scaled(workloads.BATCH_2D_FP32_256, strategy=args.strategy)
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


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


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
            # nvidia-smi takes longer to start than a few periods of a small
            # workload last
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "the timed region ended before the first sample"}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on the host: CPU baseline and the reference arm
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_period_rate(wl, n_sample, budget_s, max_periods=None, threads=1):
    """Time the FP64 oracle, as it stands, on a sample of the workload:
    n_sample initial particles, full periods until budget_s has elapsed.
    Returns the per-period times, particle-steps and the threads used."""
    import oracle
    oracle.build()
    if wl.get("dim", 2) == 4:
        o = oracle.Oracle4(hbar=wl["hbar"], mass=wl["mass"], dt=wl["dt"], Z=wl["Z"], a=wl["a"],
                           xc=wl["xc"], lam=wl["lam"], nx=wl["nx"], nk=wl["nk"],
                           xmin=wl["xmin"], xmax=wl["xmax"], kmin=wl["kmin"], kmax=wl["kmax"],
                           ny=wl["ny"], nkap=wl["nkap"], n_alpha=n_sample, seed=wl["seed"])
        used = 1
    else:
        threads = max(1, min(threads, oracle.max_threads()))
        o = oracle.Oracle(hbar=wl["hbar"], mass=wl["mass"], dt=wl["dt"], gamma0=wl["gamma0"],
                          H=wl["H"], w=wl["w"], xc=wl["xc"], nx=wl["nx"], nk=wl["nk"],
                          xmin=wl["xmin"], xmax=wl["xmax"], kmin=wl["kmin"], kmax=wl["kmax"],
                          strategy=oracle.SP1 if wl["strategy"] == "sp1" else oracle.SP2,
                          n_alpha=n_sample, seed=wl["seed"], comps=tuple(wl.get("comps", ())),
                          threads=threads)
        used = o.threads
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
    return times, psteps, used


def cpu_baseline(wl, budget_s=10.0):
    """The oracle as it stands on the host: on all cores (the reported value)
    and on one core, each on a bounded sample of the workload."""
    n = int(wl["n_alpha"])
    P = wl["resample_every"]
    cores = host_cores()
    n1 = min(n, 1_000_000)
    t1, p1, _ = oracle_period_rate(wl, n1, budget_s=budget_s)
    nall = min(n, 1_000_000 * max(1, cores // 2))
    ta, pa, used = oracle_period_rate(wl, nall, budget_s=budget_s, threads=cores)
    return {"value": sum(pa) / sum(ta), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%d of the %d particles, %d full %d-interval periods incl. annihilation, "
                      "FP64 oracle, %d threads over contiguous particle chunks"
                      % (nall, n, len(ta), P, used),
            "single_thread": {"value": sum(p1) / sum(t1), "cores": 1,
                              "sample": "%d of the %d particles, %d full periods"
                                        % (n1, n, len(t1))}}


def reference_arm(args, wl):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    cores = host_cores()
    n_sample = 200_000 * max(1, min(cores, 16))
    times, psteps, used = oracle_period_rate(wl, n_sample, budget_s=1e9,
                                             max_periods=args.warmup + args.steps,
                                             threads=cores)
    t = sum(times[args.warmup:])
    ps = sum(psteps[args.warmup:])
    value = ps / t if t > 0 else 0.0
    sample = ("%d-particle sample (of %d) of the same workload, %d-interval periods "
              "incl. annihilation, FP64 oracle, %d threads"
              % (n_sample, int(wl["n_alpha"]), wl["resample_every"], used))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
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
            "cuda_graphs": not args.no_graph,
            "parallelism": "replicas x%d" % args.gpus}


# ---------------------------------------------------------------------------
# the integer-pipe ceiling of the hot path's random numbers
# ---------------------------------------------------------------------------
def philox_ceiling(iters=4096, reps=5):
    """Chained Philox4x32-10 calls per second on every resident thread (the
    library's own call, wbrw_philox_chain), timed with CUDA events on its
    stream after warm-up: the best of `reps` launches."""
    import torch
    from paper_1709_02121_gb300 import wbrw
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nthreads = props.multi_processor_count * props.max_threads_per_multi_processor
    out = torch.empty(nthreads, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    best = 0.0
    for r in range(reps + 3):
        ev[0].record(s)
        st = wbrw.wbrw_philox_chain(0x1234 + r, iters, nthreads, out.data_ptr(), s.cuda_stream)
        if st != wbrw.OK:
            raise RuntimeError("wbrw_philox_chain failed: %d" % st)
        ev[1].record(s)
        s.synchronize()
        if r >= 3:
            best = max(best, nthreads * iters / (ev[0].elapsed_time(ev[1]) / 1e3))
    return best


# Philox4x32-10 calls the algorithm makes.  Event kernel: per candidate
# interval (its first event; in FP32 2D one call gives the life-length and
# the event's uniforms, FP32 4D draws the life-length and the event
# separately, FP64 draws the life-length and the event's two calls) and per
# first-event pair (the offspring ids).  First wave: per particle and period
# (regeneration offsets and, in FP32, the first candidate gap) and per
# particle-step (FP64 draws every interval's candidate test).
PHILOX_EVENT = {"fp32": (1, 1), "fp32_4d": (2, 1), "fp64": (3, 1), "fp64_4d": (3, 1)}
PHILOX_FIRST = {"fp32": (1, 0), "fp32_4d": (1, 0), "fp64": (1, 1), "fp64_4d": (2, 1)}
# Lane instructions of one call, read by ncu from the chained probe
# (smsp__thread_inst_executed.sum / calls; profiles/k_philox_chain_311296x4096.md).
INST_PER_PHILOX = 42.0
SMS, INT32_LANES = 152, 64
# DRAM bytes per unit measured by ncu for the plain sp1 workloads
# (profiles/); None where no capture of the current kernels exists (other
# strategies, batches, FP64, and the 2D FP32 kernels that the one-launch
# period replaced on this workload)
TRAFFIC_PER_PSTEP = {"fp32": None, "fp64": None, "fp32_4d": 1.19, "fp64_4d": None}
TRAFFIC_PER_CANDIDATE = {"fp32": None, "fp64": None, "fp32_4d": 49.2, "fp64_4d": None}
# the one-launch period: its DRAM bytes per candidate interval (the queue
# entries written by the first wave and read back by the rounds dominate)
TRAFFIC_PERIOD_PER_CANDIDATE = {"fp32": 44.2, "fp32_4d": 69.3}


def _traffic(table, wl):
    if wl.get("strategy", "sp1") != "sp1" or "instances" in wl:
        return None
    return table.get(_key(wl))
# Algorithmic HBM bytes per particle-step of the whole step if every interval
# moved the particle state through HBM (x, k read and x written, the
# offspring's share and the resampling amortised over the period): FP32 2D
# 14.5 B (sp1), + 8 B of weights read and written (sp2, wp); FP32 4D, two
# positions and two wavevectors, 28 B.
HBM_BYTES_PER_PSTEP = {"sp1": 14.5, "sp2": 22.5, "wp": 22.5, "4d": 28.0}


def _key(wl):
    return wl["precision"] + ("_4d" if wl.get("dim", 2) == 4 else "")


def _peak(ceiling, clk, peaks):
    """The Philox ceiling in Gcalls/s: the live measurement if there is one,
    and the figure derived from the unit counts and the sampled SM clock."""
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0
    derived = SMS * INT32_LANES * sm_mhz * 1e6 / INST_PER_PHILOX / 1e9
    return (ceiling / 1e9 if ceiling else derived), derived, sm_mhz


def roofline_event(wl, ev_ms, ev_n, cand, pairs, ceiling, clk, peaks):
    """Roofline of the event kernel (k_event), which performs the first event
    of every candidate interval: the kick, the acceptance and, for an
    accepted event, the pair; in FP32 the offspring then fly to the end of
    the period into the histogram inside the same kernel.

    achieved = the Philox4x32-10 calls the algorithm makes for the timed
    region's candidate intervals and first-event pairs (device counters) /
    the kernel's summed CUDA-event time.
    peak = the chained-Philox ceiling measured on this GPU in the same run."""
    if not ev_n or ev_ms <= 0 or cand <= 0:
        return None
    a, b = PHILOX_EVENT[_key(wl)]
    peak, derived, sm_mhz = _peak(ceiling, clk, peaks)
    calls = a * cand + b * pairs
    ach = calls / (ev_ms / 1e3) / 1e9
    tpc = _traffic(TRAFFIC_PER_CANDIDATE, wl)
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gcalls/s",
            "frac": ach / peak, "traffic": tpc and tpc * cand / ev_n,
            "kernel": "k_event<%s%s,bin>" % (wl["precision"],
                                             ",4d" if wl.get("dim", 2) == 4 else ""),
            "launch_ms": ev_ms / ev_n, "launches": ev_n, "total_ms": ev_ms,
            "candidates_per_launch": cand / ev_n, "first_pairs_per_candidate": pairs / cand,
            "philox_calls_per_candidate": calls / cand,
            "peak_derived": derived,
            "peak_basis": "Philox4x32-10 calls/s of the chained probe measured in this run "
                          "(derived: %d SM x %d INT32 lanes x %.0f MHz / %.1f lane instructions "
                          "per call)" % (SMS, INT32_LANES, sm_mhz, INST_PER_PHILOX)}


def roofline(wl, kern_ms, kern_n, psteps_first, ceiling, clk, peaks):
    """Roofline of the first wave: the fused regenerate + flight + histogram
    pass that carries the particles present at the start of each period.
    The particle state never leaves registers and HBM sees only the
    candidate queue, so the pass is bound by the integer pipe.

    achieved = the Philox calls the algorithm makes per first-wave particle
    and period (PHILOX_FIRST) x the particles of one launch / the launch's
    average CUDA-event time.
    peak = the chained-Philox ceiling measured on this GPU in the same run."""
    if not kern_n or kern_ms <= 0:
        return None
    R = wl["resample_every"]
    base, per_interval = PHILOX_FIRST[_key(wl)]
    per_pstep = (base + per_interval * R) / R
    per_launch_ms = kern_ms / kern_n
    peak, derived, sm_mhz = _peak(ceiling, clk, peaks)
    ach = per_pstep * (psteps_first / kern_n) / (per_launch_ms / 1e3) / 1e9
    tpp = _traffic(TRAFFIC_PER_PSTEP, wl)
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gcalls/s",
            "frac": ach / peak, "traffic": tpp and tpp * psteps_first / kern_n,
            "kernel": "k_flight<%s%s,regen,bin>" % (wl["precision"],
                                                     ",4d" if wl.get("dim", 2) == 4 else ""),
            "launch_ms": per_launch_ms, "launches": kern_n, "total_ms": kern_ms,
            "first_wave_particle_steps_per_launch": psteps_first / kern_n,
            "philox_calls_per_particle_step": per_pstep,
            "peak_derived": derived,
            "peak_basis": "Philox4x32-10 calls/s of the chained probe measured in this run "
                          "(derived: %d SM x %d INT32 lanes x %.0f MHz / %.1f lane instructions "
                          "per call)" % (SMS, INT32_LANES, sm_mhz, INST_PER_PHILOX)}


def hbm_equivalent(wl, value, peaks):
    """The whole step's rate as HBM bandwidth, had every interval moved the
    particle state through HBM (the bytes per particle-step above), against
    the measured copy bandwidth."""
    key = "4d" if wl.get("dim", 2) == 4 else wl["strategy"]
    b = HBM_BYTES_PER_PSTEP.get(key)
    hbm = peaks.get("hbm_gbs")
    if wl["precision"] != "fp32" or b is None or not hbm:
        return None
    ach = value * b / 1e9
    return {"bytes_per_particle_step": b, "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}


def dominant(*roofs):
    """The rooflines ordered by the kernel's total time in the timed region:
    (the dominant kernel's, the other's)."""
    r = sorted((x for x in roofs if x), key=lambda x: -x["total_ms"])
    return (r[0] if r else None), (r[1] if len(r) > 1 else None)


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


# ---------------------------------------------------------------------------
# timing of one context
# ---------------------------------------------------------------------------
def warm_up(sim, args, P, warmup):
    """`warmup` untimed periods: warmup - 1, the launch-shape autotuning
    (which releases the period graphs), then profiling on and the last one,
    which captures the period graph again with the profiling events, so that
    no capture falls in the timed region.  Profiling stays on until the end
    (switching it captures the graphs again)."""
    from paper_1709_02121_gb300 import wbrw
    for _ in range(max(warmup - 1, 0)):
        sim.run(P)
    tuning = autotune(sim, args)
    wbrw.wbrw_profile(sim.ctx, True)
    sim.run(P)
    return tuning


def autotune(sim, args):
    """Pick the launch shape by timing one period under each (results do not
    depend on it); the run continues from where it was."""
    if getattr(args, "tuning", ""):
        b, p = (int(v) for v in args.tuning.split(","))
        b, p = sim.tuning(b, p)
        return {"blocks_per_sm": b, "event_passes": p, "autotuned": False}
    if args.no_autotune:
        b, p = sim.tuning()
        return {"blocks_per_sm": b, "event_passes": p, "autotuned": False}
    (b, p), table = sim.autotune(trials=2)
    return {"blocks_per_sm": b, "event_passes": p, "autotuned": True,
            "period_ms": [[round(float(v), 4) for v in row] for row in table]}


def _barrier():
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()


def timed_periods(sim, P, steps, flush, local):
    """`steps` periods, each bracketed by CUDA events on the context's stream,
    the L2 flushed before each; clocks sampled meanwhile; a barrier and a
    device synchronisation on both sides.  Returns the summed device time,
    the counters before and after, the profiling reads and the clock
    record."""
    import torch
    from paper_1709_02121_gb300 import wbrw
    stream = sim.stream
    _barrier()
    c0 = sim.counters()
    wbrw.wbrw_profile(sim.ctx, True)  # clears what the last warm-up period recorded
    clocks = Clocks(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i)  # evict the histogram and plan from L2
        stream.wait_stream(torch.cuda.current_stream())  # the flush ends before the timing starts
        starts[i].record(stream)
        sim.run(P)
        ends[i].record(stream)
    _barrier()
    clk = clocks.stop()
    kern = wbrw.wbrw_profile_read(sim.ctx)
    ev = wbrw.wbrw_profile_read_events(sim.ctx)
    c1 = sim.counters()
    t_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    return t_ms, c0, c1, kern, ev, clk


def rooflines(wl, c0, c1, kern, ev, ceiling, clk, peaks):
    d = {k: c1[k] - c0[k] for k in ("particle_steps_first", "candidates", "first_pairs")}
    if not ev[1] and kern[1]:  # one launch per period: the first wave and the rounds fused
        return roofline_period(wl, kern[0], kern[1], d["particle_steps_first"], d["candidates"],
                               d["first_pairs"], ceiling, clk, peaks), None
    return dominant(
        roofline(wl, kern[0], kern[1], d["particle_steps_first"], ceiling, clk, peaks),
        roofline_event(wl, ev[0], ev[1], d["candidates"], d["first_pairs"], ceiling, clk, peaks))


def roofline_period(wl, ms, n, psteps_first, cand, pairs, ceiling, clk, peaks):
    """Roofline of the one-launch period (k_period): the first wave and every
    event round in one kernel.  achieved = the first wave's Philox calls
    (PHILOX_FIRST per first-wave particle-step) + the event calls
    (PHILOX_EVENT per candidate and per first-event pair) / the launches'
    summed CUDA-event time; peak = the chained-Philox ceiling."""
    if not n or ms <= 0:
        return None
    key = _key(wl)
    R = wl["resample_every"]
    base, per_interval = PHILOX_FIRST[key]
    a, b = PHILOX_EVENT[key]
    calls = (base + per_interval * R) / R * psteps_first + a * cand + b * pairs
    peak, derived, sm_mhz = _peak(ceiling, clk, peaks)
    ach = calls / (ms / 1e3) / 1e9
    t = _traffic(TRAFFIC_PERIOD_PER_CANDIDATE, wl)
    traffic = t * cand / n if t is not None else None
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gcalls/s",
            "frac": ach / peak, "traffic": traffic,
            "kernel": "k_period<%s%s>" % (wl["precision"], ",4d" if wl.get("dim", 2) == 4 else ""),
            "launch_ms": ms / n, "launches": n, "total_ms": ms,
            "first_wave_particle_steps_per_launch": psteps_first / n,
            "candidates_per_launch": cand / n, "first_pairs_per_candidate": pairs / max(cand, 1),
            "philox_calls_per_launch": calls / n, "peak_derived": derived,
            "peak_basis": "Philox4x32-10 calls/s of the chained probe measured in this run "
                          "(derived: %d SM x %d INT32 lanes x %.0f MHz / %.1f lane instructions "
                          "per call)" % (SMS, INT32_LANES, sm_mhz, INST_PER_PHILOX)}


def e2e_same_periods(sim, wl, P, steps, ckpt):
    """End to end through the C ABI over the very periods the device-timed
    region ran: starting from the host checkpoint taken before it, each step
    restores the histogram from pinned host memory, runs one period, and
    reads back the histogram and the observables.  The run is a function of
    the checkpoint, so these are the same periods (their particle-steps are
    compared with the timed region's)."""
    import torch
    from paper_1709_02121_gb300 import wbrw
    grid_h, step, epoch = ckpt
    # the observables are read into pinned host memory too
    dens_h = torch.empty(wl["nx"] * wl["nk"], dtype=torch.float64).pin_memory()
    marg_h = torch.empty(wl["nx"], dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    pe0 = sim.counters()["particle_steps"]
    t0 = time.perf_counter()
    T_last = None
    for _ in range(steps):
        sim.restore(grid_h.numpy(), step, epoch)
        sim.run(P)
        _, step, epoch = sim.checkpoint(grid_h.numpy())
        if getattr(sim, "ninst", 1) > 1:
            T_last = float(sim.transmissions().mean())
        else:
            _, _, T_last, _ = wbrw.wbrw_density(sim.ctx, wl["nx"], wl["nk"], dens_h.numpy(),
                                                marg_h.numpy())
    te = time.perf_counter() - t0
    pe = sim.counters()["particle_steps"] - pe0
    return pe / te, pe, T_last


def measure(args, wl, sim, steps, warmup, local, flush, ceiling, peaks, e2e_bytes=None):
    """Warm up, autotune and time `steps` periods of a context; optionally
    repeat them end to end.  Returns the measurement as a dict."""
    import torch
    P = wl["resample_every"]
    tuning = warm_up(sim, args, P, warmup)
    ckpt = None
    if e2e_bytes is not None:
        shape = sim.grid_counts().shape
        grid_h = torch.empty(shape, dtype=torch.int32).pin_memory()
        _, step, epoch = sim.checkpoint(grid_h.numpy())
        ckpt = (grid_h, step, epoch)
    t_ms, c0, c1, kern, ev, clk = timed_periods(sim, P, steps, flush, local)
    psteps = c1["particle_steps"] - c0["particle_steps"]
    roof, roof2 = rooflines(wl, c0, c1, kern, ev, ceiling, clk, peaks)
    out = {"t_ms": t_ms, "psteps": psteps, "launches": c1["launches"] - c0["launches"],
           "live_end": c1["live"], "roofline": roof, "roofline_secondary": roof2,
           "clocks": clk, "tuning": tuning, "e2e": None}
    if ckpt is not None:
        rate, pe, T_last = e2e_same_periods(sim, wl, P, steps, ckpt)
        h2d, d2h = e2e_bytes
        out["e2e"] = {"value": rate, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "steps": steps,
                      "same_periods_as_value": pe == psteps,
                      "transmission_last": T_last}
    return out


def summary(wl, m, steps, peaks):
    """The compact record of a secondary measurement."""
    value = m["psteps"] / (m["t_ms"] / 1e3)
    return {"workload": wl["name"], "value": value, "unit": UNIT,
            "ms_per_step": m["t_ms"] / steps, "steps": steps,
            "particle_steps": m["psteps"], "roofline": m["roofline"],
            "roofline_secondary": m["roofline_secondary"],
            "hbm_equivalent": hbm_equivalent(wl, value, peaks), "clocks": m["clocks"],
            "tuning": {k: v for k, v in (m["tuning"] or {}).items() if k != "period_ms"},
            "gpu_launches": m["launches"]}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _setup(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1709_02121_gb300 import build
    build.build()
    return ws, rank, local


def _free(*objs):
    import torch
    for o in objs:
        if o is not None:
            o.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def ours(args, wl):
    import torch
    import torch.distributed as dist
    ws, rank, local = _setup(args)
    from paper_1709_02121_gb300 import Simulation, Simulation4

    peaks = load_peaks()
    ceiling = philox_ceiling()
    wl = workloads.scaled(wl, seed=wl["seed"] + rank)
    n = int(wl["n_alpha"])
    cap = int(args.capacity_factor * n) + (1 << 20)
    model = Simulation4 if wl.get("dim", 2) == 4 else Simulation
    sim = model(wl, capacity=cap, stream=torch.cuda.Stream())
    if not args.no_graph:
        sim.graph(True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    cells = sim.cells
    e2e_bytes = None if args.no_e2e else (
        cells * 4, cells * 4 + wl["nx"] * wl["nk"] * 8 + wl["nx"] * 8 + 16)
    m = measure(args, wl, sim, args.steps, args.warmup, local, flush, ceiling, peaks, e2e_bytes)
    _free(sim)
    del sim

    t_max, ps_all, e2e_sum = reduce_over_ranks(ws, m["t_ms"], m["psteps"],
                                               m["e2e"]["value"] if m["e2e"] else 0.0, "cuda")
    if m["e2e"] is not None:
        m["e2e"]["value"] = e2e_sum
    secondary = None
    if (ws == 1 and not args.no_secondary and args.workload == "gauss2d_fp32_n1e8"
            and wl["strategy"] == "sp1" and not args.particles):
        secondary = secondaries(args, local, flush, ceiling, peaks)
    if rank == 0:
        value = ps_all / (t_max / 1e3)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if wl["precision"] == "fp32" else "f64",
                "data": "synthetic", "config": config_of(wl, args),
                "e2e": m["e2e"], "gpu_launches": m["launches"], "roofline": m["roofline"],
                "roofline_secondary": m["roofline_secondary"],
                "hbm_equivalent": hbm_equivalent(wl, value, peaks),
                "philox_ceiling_calls_per_s": ceiling,
                "clocks": m["clocks"], "tuning": m["tuning"],
                "live_particles_end": m["live_end"], "particle_steps": m["psteps"]}
        if secondary:
            line["secondary"] = secondary
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def secondaries(args, local, flush, ceiling, peaks):
    """The other parts of the metric, each measured like the default line
    (warm-up, autotuning, CUDA events, L2 flush, clocks) over fewer periods."""
    import torch
    from paper_1709_02121_gb300 import Simulation, Simulation4
    W, K = 3, 6

    def plain_like(wl, model, graphs):
        n = int(wl["n_alpha"])
        sim = model(wl, capacity=int(args.capacity_factor * n) + (1 << 20),
                    stream=torch.cuda.Stream())
        try:
            if graphs:
                sim.graph(True)
            m = measure(args, wl, sim, K, W, local, flush, ceiling, peaks)
        finally:
            _free(sim)
        res = summary(wl, m, K, peaks)
        res["cuda_graphs"] = graphs
        return res

    jobs = [
        # sp2: the 1e8 workload with the signed bootstrap filter
        ("sp2", lambda: plain_like(workloads.scaled(workloads.GAUSS_2D_FP32_1E8, strategy="sp2"),
                                   Simulation, not args.no_graph)),
        # the FP64 parity path at its own size (2e5 particles, 240 x 128 cells, dt = 0.1)
        ("fp64", lambda: plain_like(workloads.scaled(workloads.GAUSS_2D_FP64_2E5), Simulation,
                                    not args.no_graph)),
        # the 4D Helium-like system
        ("he4d", lambda: plain_like(workloads.scaled(workloads.HE_4D_FP32_5E7), Simulation4,
                                    not args.no_graph)),
        # the batch of 256 against the plain per-instance path
        ("batch", lambda: _strip(batch_measure(args, workloads.BATCH_2D_FP32_256, K, W, local,
                                               flush, ceiling, peaks, plain=True))),
        # the same batch with the signed bootstrap (every instance filtered on its own)
        ("batch_sp2", lambda: _strip(batch_measure(
            args, workloads.scaled(workloads.BATCH_2D_FP32_256, strategy="sp2"), K, W, local,
            flush, ceiling, peaks, plain=True))),
        # the gradient of T(H, w) at the 64 points against the forward run
        ("grad", lambda: grad_measure(args, workloads.GRAD_2D_FP32_64, local, flush, ceiling,
                                      peaks, group=4, points=64)),
    ]
    out = {}
    for name, job in jobs:
        # a failure here must not cost the default line: it is recorded
        try:
            out[name] = job()
        except Exception as e:  # noqa: BLE001
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
    return out


def batch_measure(args, spec, steps, warmup, local, flush, ceiling, peaks, plain=True,
                  e2e=False, seed_offset=0):
    """The batched workload: all instances in one context and the same
    launches, timed like the plain workload; then the plain per-instance path
    (one context per instance, run one after the other on the same GPU) for
    the same periods, for comparison."""
    import numpy as np
    import torch
    from paper_1709_02121_gb300 import Batch, Simulation, wbrw

    wl = workloads.scaled(spec, seed=spec["seed"] + seed_offset)
    insts = workloads.batch_instances(wl, args.n_scale)
    n_total = sum(v["n_init"] for v in insts)
    cap = int(args.capacity_factor * n_total) + (1 << 20)
    sim = Batch(wl, insts, capacity=cap, stream=torch.cuda.Stream())
    graphs = not args.no_graph
    if graphs:
        sim.graph(True)
    m_cells = len(insts) * wl["nx"] * wl["nk"]
    m = measure(args, wl, sim, steps, warmup, local, flush, ceiling, peaks,
                (m_cells * 4, m_cells * 4 + len(insts) * 8) if e2e else None)
    T_batch = sim.transmissions()
    _free(sim)
    del sim
    res = summary(wl, m, steps, peaks)
    ns = [v["n_init"] for v in insts]
    res.update({"instances": len(insts), "particles": int(n_total),
                "particles_min_max": [min(ns), max(ns)], "cuda_graphs": graphs,
                "transmission_mean": float(np.mean(T_batch)), "e2e": m["e2e"],
                "live_end": m["live_end"], "_m": m})
    if plain:
        # one context per instance on shared buffers sized for the largest
        # instance, the same warm-up and timed periods, device time summed
        # over the instances' timed periods
        P = wl["resample_every"]
        nmax = max(ns)
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
            for _ in range(warmup):
                wbrw.wbrw_run(ctx, P)
            p0 = wbrw.wbrw_counters(ctx)["particle_steps"]
            flush.fill_(0)
            host.stream.wait_stream(torch.cuda.current_stream())
            ev[0].record(host.stream)
            for _ in range(steps):
                wbrw.wbrw_run(ctx, P)
            ev[1].record(host.stream)
            torch.cuda.synchronize()
            t_plain += ev[0].elapsed_time(ev[1])
            ps_plain += wbrw.wbrw_counters(ctx)["particle_steps"] - p0
            wbrw.wbrw_destroy(ctx)
        del host
        torch.cuda.empty_cache()
        res["plain_per_instance"] = {
            "value": ps_plain / (t_plain / 1e3), "unit": UNIT, "ms_per_step": t_plain / steps,
            "particle_steps": ps_plain,
            "path": "one context per instance, instances one after the other",
            "cuda_graphs": graphs}
        res["speedup_vs_plain"] = (t_plain / steps) / res["ms_per_step"]
    return res


def grad_measure(args, spec, local, flush, ceiling, peaks, group=4, points=64,
                 seed_offset=0):
    """The differentiation workload: T(H, w) and its likelihood-ratio
    derivatives at `points` of the 64 parameter points, `group` per batch.
    Each batch runs the whole t = 20 (the first three periods untimed) twice:
    forward (no tangents) and gradient (tangent mode, the replay that
    autograd's backward runs); the two must give the same T."""
    import numpy as np
    import torch
    from paper_1709_02121_gb300 import Batch, wbrw

    wl = workloads.scaled(spec, seed=spec["seed"] + seed_offset)
    pts = workloads.grad_points(wl)
    if points < len(pts):
        idx = np.linspace(0, len(pts) - 1, points).round().astype(int)
        pts = [pts[i] for i in idx]
    n = max(1, int(round(wl["n_per_point"] * args.n_scale)))
    P = wl["resample_every"]
    periods = wl["steps"] // P
    W = 3
    K = periods - W
    tot = {False: [0.0, 0, 0], True: [0.0, 0, 0]}
    clk_all, T_all, G_all = [], [], []
    for g0 in range(0, len(pts), group):
        chunk = pts[g0:g0 + group]
        insts = [dict(H=h, w=v, xc=wl["xc"], x0=wl["x0"], sigma_x=wl["sigma_x"], k0=wl["k0"],
                      n_init=n, n_alpha=n) for h, v in chunk]
        cap = int(args.capacity_factor * n * len(insts)) + (1 << 20)
        Ts = {}
        for tangent in (False, True):
            b = Batch(dict(wl, tangent=tangent), insts, cap, stream=torch.cuda.Stream())
            if not args.no_graph:
                b.graph(True)
            for _ in range(W - 1):
                b.run(P)
            # profiling on before the last warm-up period, which captures
            # the period graph with its events outside the timed region
            wbrw.wbrw_profile(b.ctx, True)
            b.run(P)
            t_ms, c0, c1, _, _, clk = timed_periods(b, P, K, flush, local)
            tot[tangent][0] += t_ms
            tot[tangent][1] += c1["particle_steps"] - c0["particle_steps"]
            tot[tangent][2] += c1["launches"] - c0["launches"]
            Ts[tangent] = b.transmissions()
            if tangent:
                G_all.append(b.transmission_gradients())
                clk_all.append(clk)
            _free(b)
            del b
        if not np.array_equal(Ts[False], Ts[True]):
            raise RuntimeError("the tangent run did not reproduce the forward run")
        T_all.append(Ts[True])
    fwd_ms, fwd_ps, _ = tot[False]
    bwd_ms, bwd_ps, bwd_launch = tot[True]
    G = np.concatenate(G_all)
    clk = next((c for c in clk_all if c), None)
    return {"workload": wl["name"], "value": bwd_ps / (bwd_ms / 1e3), "unit": UNIT,
            "points": len(pts), "points_per_batch": group, "particles_per_point": n,
            "dt": wl["dt"], "t_end": wl["steps"] * wl["dt"], "intervals_per_step": P,
            "timed_periods_per_batch": K, "ms_per_period_of_a_batch": bwd_ms / (K * len(T_all)),
            "particle_steps": bwd_ps, "gpu_launches": bwd_launch, "clocks": clk,
            "forward": {"value": fwd_ps / (fwd_ms / 1e3), "unit": UNIT,
                        "ms_per_period_of_a_batch": fwd_ms / (K * len(T_all))},
            "gradient_cost_vs_forward": bwd_ms / fwd_ms,
            "lr_speedup_vs_central_differences": 4.0 * fwd_ms / bwd_ms,
            "note": "value: the gradient run (tangent mode), whose particle-steps include the "
                    "sign-0 tangent particles; T and dT/dtheta at t_end for every point",
            "T": [round(float(x), 5) for x in np.concatenate(T_all)],
            "dT_dH": [round(float(x), 5) for x in G[:, 0]],
            "dT_dw": [round(float(x), 5) for x in G[:, 1]]}


def _strip(res):
    return {k: v for k, v in res.items() if not k.startswith("_")}


def ours_batch(args, spec):
    """The batched workload as the line's own workload."""
    import torch
    import torch.distributed as dist
    ws, rank, local = _setup(args)
    peaks = load_peaks()
    ceiling = philox_ceiling()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    res = batch_measure(args, spec, args.steps, args.warmup, local, flush, ceiling, peaks,
                        plain=not args.no_plain, e2e=not args.no_e2e, seed_offset=rank)
    m = res["_m"]
    e2e = m["e2e"]
    t_max, ps_all, e2e_sum = reduce_over_ranks(ws, m["t_ms"], m["psteps"],
                                               e2e["value"] if e2e else 0.0, "cuda")
    if e2e is not None:
        e2e["value"] = e2e_sum
    if rank == 0:
        value = ps_all / (t_max / 1e3)
        wl = workloads.scaled(spec)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": wl["name"], "instances": res["instances"],
                           "particles": res["particles"],
                           "particles_min_max": res["particles_min_max"],
                           "grid_per_instance": [wl["nx"], wl["nk"]], "dt": wl["dt"],
                           "intervals_per_step": wl["resample_every"],
                           "strategy": wl["strategy"],
                           "precision": "fp32", "cuda_graphs": res["cuda_graphs"],
                           "l2": "flushed (512 MiB write) between timed steps",
                           "parallelism": "replicas x%d" % ws},
                "e2e": e2e, "gpu_launches": m["launches"], "roofline": m["roofline"],
                "roofline_secondary": m["roofline_secondary"],
                "hbm_equivalent": hbm_equivalent(wl, value, peaks),
                "philox_ceiling_calls_per_s": ceiling, "clocks": m["clocks"],
                "tuning": m["tuning"], "live_particles_end": m["live_end"],
                "particle_steps": m["psteps"], "transmission_mean": res["transmission_mean"]}
        if "plain_per_instance" in res:
            line["plain_per_instance"] = res["plain_per_instance"]
            line["speedup_vs_plain"] = res["speedup_vs_plain"]
        if not args.no_cpu_baseline and ws == 1:
            v = workloads.batch_instances(wl, args.n_scale)[0]
            one = workloads.scaled(wl, H=v["H"], w=v["w"], k0=v["k0"], n_alpha=v["n_init"])
            cb = cpu_baseline(one)
            cb["sample"] = "instance 0 (H=%.3g, w=%.3g, k0=%.3g): " % (
                v["H"], v["w"], v["k0"]) + cb["sample"]
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def ours_grad(args, spec):
    """The differentiation workload as the line's own workload."""
    import torch
    import torch.distributed as dist
    ws, rank, local = _setup(args)
    peaks = load_peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    res = grad_measure(args, spec, local, flush, None, peaks, group=args.group,
                       points=args.points, seed_offset=rank)
    t_ms = res["particle_steps"] / res["value"] * 1e3
    t_max, ps_all, _ = reduce_over_ranks(ws, t_ms, res["particle_steps"], 0.0, "cuda")
    if rank == 0:
        wl = workloads.scaled(spec)
        value = ps_all / (t_max / 1e3)
        nb = -(-res["points"] // res["points_per_batch"])
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": res["timed_periods_per_batch"] * nb, "warmup": 3 * nb,
                "ms_per_step": res["ms_per_period_of_a_batch"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (f32 tangent weights)", "data": "synthetic",
                "config": {"workload": wl["name"], "points": res["points"],
                           "points_per_batch": res["points_per_batch"],
                           "particles_per_point": res["particles_per_point"],
                           "grid": [wl["nx"], wl["nk"]], "dt": wl["dt"],
                           "t_end": res["t_end"], "intervals_per_step": wl["resample_every"],
                           "strategy": "sp1", "precision": "fp32 state and tangent weights",
                           "cuda_graphs": not args.no_graph,
                           "l2": "flushed (512 MiB write) between timed steps",
                           "parallelism": "replicas x%d" % ws},
                "e2e": None, "gpu_launches": res["gpu_launches"], "clocks": res["clocks"]}
        line.update({k: res[k] for k in ("particle_steps", "note", "forward",
                                          "gradient_cost_vs_forward",
                                          "lr_speedup_vs_central_differences", "T", "dT_dH",
                                          "dT_dw")})
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


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
