"""Host logic of bench.py that needs no GPU: the roofline arithmetic of the
first wave and the workload selection."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.path.insert(0, ROOT)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_counts_the_algorithmic_operations(bench):
    wl = {"precision": "fp32", "resample_every": 10}
    r = bench.roofline(wl, kern_ms=4.0, kern_n=2, psteps_first=3.2e9, peaks={},
                       clk={"sm_mhz": 2070.0})
    # 120 integer operations per particle and 10-interval period: 12 per
    # particle-step; 1.6e9 particle-steps in 2 ms per launch
    assert r["int_ops_per_particle_step"] == pytest.approx(12.0)
    assert r["achieved"] == pytest.approx(12.0 * 1.6e9 / 2e-3 / 1e9)
    assert r["peak"] == pytest.approx(152 * 64 * 2070e6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["launch_ms"] == pytest.approx(2.0)
    # the traffic per launch scales the measured bytes per particle-step
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_PSTEP["fp32"] * 1.6e9)


def test_roofline_of_the_fp64_and_4d_paths(bench):
    r = bench.roofline({"precision": "fp64", "resample_every": 10}, 1.0, 1, 1e6, {},
                       {"sm_mhz": 2000.0})
    # one Philox per interval plus the regeneration call and the decode
    assert r["int_ops_per_particle_step"] == pytest.approx((116 + 100 * 10) / 10)
    assert r["traffic"] is None
    r4 = bench.roofline({"precision": "fp32", "dim": 4, "resample_every": 16}, 1.0, 1, 1e6,
                        {}, {"sm_mhz": 2000.0})
    assert r4["int_ops_per_particle_step"] == pytest.approx(135 / 16)
    assert r4["kernel"] == "k_flight<fp32,4d,regen,bin>"
    assert bench.roofline({"precision": "fp32", "resample_every": 10}, 0.0, 0, 0, {}, {}) is None


def test_workload_selection(bench):
    class A:
        workload = "gauss2d_fp32_n1e8"
        strategy = "sp2"
        particles = 0
    wl = bench.workload(A)
    assert wl["n_alpha"] == 100_000_000 and wl["strategy"] == "sp2"
    A.particles = 1.5e7
    assert bench.workload(A)["n_alpha"] == 15_000_000
    A.workload, A.particles = "he4d_fp32_n5e7", 0
    assert bench.workload(A)["dim"] == 4


def test_event_roofline_counts_candidates_and_pairs(bench):
    wl = {"precision": "fp32", "resample_every": 10}
    r = bench.roofline_event(wl, ev_ms=3.0, ev_n=10, cand=2e8, pairs=1.2e8, peaks={},
                             clk={"sm_mhz": 2000.0})
    # 120 operations per candidate and 140 per pair over the summed 3 ms
    assert r["achieved"] == pytest.approx((120 * 2e8 + 140 * 1.2e8) / 3e-3 / 1e9)
    assert r["peak"] == pytest.approx(152 * 64 * 2000e6 / 1e9)
    assert r["launch_ms"] == pytest.approx(0.3) and r["total_ms"] == pytest.approx(3.0)
    assert r["candidates_per_launch"] == pytest.approx(2e7)
    assert r["first_pairs_per_candidate"] == pytest.approx(0.6)
    assert r["kernel"] == "k_event<fp32,bin>" and r["bound"] == "alu"
    tpc = bench.TRAFFIC_PER_CANDIDATE["fp32"]
    assert r["traffic"] == (None if tpc is None else pytest.approx(tpc * 2e7))
    assert bench.roofline_event(wl, 0.0, 0, 0, 0, {}, {}) is None


def test_the_dominant_kernel_is_the_one_with_more_time(bench):
    wl = {"precision": "fp32", "resample_every": 10}
    first = bench.roofline(wl, kern_ms=2.0, kern_n=2, psteps_first=3.2e9, peaks={},
                           clk={"sm_mhz": 2070.0})
    ev = bench.roofline_event(wl, 3.0, 20, 2e8, 1.2e8, {}, {"sm_mhz": 2070.0})
    assert bench.dominant(first, ev) == (ev, first)
    assert bench.dominant(ev, None) == (ev, None)
    assert bench.dominant(None, None) == (None, None)


def test_warm_up_switches_profiling_on_before_its_last_period(bench, monkeypatch):
    """The period graph is captured again when profiling is switched on, so
    the switch happens before the last warm-up period: no capture falls in
    the timed region."""
    from paper_1709_02121_gb300 import wbrw
    calls = []

    class Sim:
        ctx = object()

        def run(self, n):
            calls.append(("run", n))

    monkeypatch.setattr(wbrw, "wbrw_profile", lambda ctx, on=True: calls.append(("profile", on)))
    monkeypatch.setattr(bench, "autotune", lambda sim, args: calls.append(("autotune",)) or {})

    class A:
        warmup = 4
    bench.warm_up(Sim(), A, 10)
    assert calls == [("run", 10)] * 3 + [("autotune",), ("profile", True), ("run", 10)]
