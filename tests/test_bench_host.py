"""Host logic of bench.py that needs no GPU: the roofline arithmetic of the
first wave and the event kernel, the HBM-equivalent rate, the CPU baseline's
arms and the workload selection."""
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


def test_first_wave_roofline_counts_philox_calls(bench):
    wl = {"precision": "fp32", "resample_every": 10}
    r = bench.roofline(wl, kern_ms=4.0, kern_n=2, psteps_first=3.2e9, ceiling=5e11,
                       clk={"sm_mhz": 2070.0}, peaks={})
    # one call per particle and 10-interval period: 0.1 per particle-step;
    # 1.6e9 particle-steps in 2 ms per launch
    assert r["philox_calls_per_particle_step"] == pytest.approx(0.1)
    assert r["achieved"] == pytest.approx(0.1 * 1.6e9 / 2e-3 / 1e9)
    assert r["unit"] == "Gcalls/s"
    assert r["peak"] == pytest.approx(500.0)           # the measured ceiling
    assert r["peak_derived"] == pytest.approx(152 * 64 * 2070e6 / 42.0 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["launch_ms"] == pytest.approx(2.0)
    # the traffic per launch scales the measured bytes per particle-step;
    # null where no capture of the kernel exists
    tpp = bench.TRAFFIC_PER_PSTEP["fp32"]
    assert r["traffic"] == (None if tpp is None else pytest.approx(tpp * 1.6e9))
    r4 = bench.roofline({"precision": "fp32", "dim": 4, "resample_every": 10}, 4.0, 2, 3.2e9,
                        None, {"sm_mhz": 2070.0}, {})
    assert r4["traffic"] == pytest.approx(bench.TRAFFIC_PER_PSTEP["fp32_4d"] * 1.6e9)
    # without a measurement the derived ceiling is the peak
    r0 = bench.roofline(wl, 4.0, 2, 3.2e9, None, {"sm_mhz": 2070.0}, {})
    assert r0["peak"] == pytest.approx(r0["peak_derived"])


def test_first_wave_roofline_of_the_fp64_and_4d_paths(bench):
    r = bench.roofline({"precision": "fp64", "resample_every": 10}, 1.0, 1, 1e6, None,
                       {"sm_mhz": 2000.0}, {})
    # the regeneration call plus one call per interval
    assert r["philox_calls_per_particle_step"] == pytest.approx((1 + 10) / 10)
    assert r["traffic"] is None
    r4 = bench.roofline({"precision": "fp32", "dim": 4, "resample_every": 16}, 1.0, 1, 1e6,
                        None, {"sm_mhz": 2000.0}, {})
    assert r4["philox_calls_per_particle_step"] == pytest.approx(1 / 16)
    assert r4["kernel"] == "k_flight<fp32,4d,regen,bin>"
    assert bench.roofline({"precision": "fp32", "resample_every": 10}, 0.0, 0, 0, None, {},
                          {}) is None


def test_event_roofline_counts_candidates_and_pairs(bench):
    wl = {"precision": "fp32", "resample_every": 10}
    r = bench.roofline_event(wl, ev_ms=3.0, ev_n=10, cand=2e8, pairs=1.2e8, ceiling=4.8e11,
                             clk={"sm_mhz": 2000.0}, peaks={})
    # one call per candidate (life-length and event) and one per pair (ids)
    assert r["achieved"] == pytest.approx((2e8 + 1.2e8) / 3e-3 / 1e9)
    assert r["philox_calls_per_candidate"] == pytest.approx(1.6)
    assert r["peak"] == pytest.approx(480.0)
    assert r["launch_ms"] == pytest.approx(0.3) and r["total_ms"] == pytest.approx(3.0)
    assert r["candidates_per_launch"] == pytest.approx(2e7)
    assert r["first_pairs_per_candidate"] == pytest.approx(0.6)
    assert r["kernel"] == "k_event<fp32,bin>" and r["bound"] == "alu"
    tpc = bench.TRAFFIC_PER_CANDIDATE["fp32"]
    assert r["traffic"] == (None if tpc is None else pytest.approx(tpc * 2e7))
    r4 = bench.roofline_event({"precision": "fp32", "dim": 4, "resample_every": 10}, 3.0, 10,
                              2e8, 1.2e8, None, {"sm_mhz": 2000.0}, {})
    assert r4["philox_calls_per_candidate"] == pytest.approx(2.6)
    assert bench.roofline_event(wl, 0.0, 0, 0, 0, None, {}, {}) is None


def test_hbm_equivalent_rate(bench):
    peaks = {"hbm_gbs": 6786.2}
    wl = {"precision": "fp32", "strategy": "sp1"}
    h = bench.hbm_equivalent(wl, 4e11, peaks)
    assert h["achieved"] == pytest.approx(4e11 * 14.5 / 1e9)
    assert h["frac"] == pytest.approx(4e11 * 14.5 / 1e9 / 6786.2)
    assert bench.hbm_equivalent(dict(wl, strategy="sp2"), 1e11, peaks)["bytes_per_particle_step"] \
        == pytest.approx(22.5)
    assert bench.hbm_equivalent(dict(wl, dim=4), 1e11, peaks)["bytes_per_particle_step"] \
        == pytest.approx(28.0)
    assert bench.hbm_equivalent(dict(wl, precision="fp64"), 1e11, peaks) is None
    assert bench.hbm_equivalent(wl, 1e11, {}) is None


def test_the_dominant_kernel_is_the_one_with_more_time(bench):
    wl = {"precision": "fp32", "resample_every": 10}
    first = bench.roofline(wl, 2.0, 2, 3.2e9, None, {"sm_mhz": 2070.0}, {})
    ev = bench.roofline_event(wl, 3.0, 20, 2e8, 1.2e8, None, {"sm_mhz": 2070.0}, {})
    assert bench.dominant(first, ev) == (ev, first)
    assert bench.dominant(ev, None) == (ev, None)
    assert bench.dominant(None, None) == (None, None)


def test_cpu_baseline_has_an_all_cores_and_a_single_thread_arm(bench, monkeypatch):
    seen = []

    def fake(wl, n, budget_s, max_periods=None, threads=1):
        seen.append((n, threads))
        return [1.0, 1.0], [10 * n * threads, 10 * n * threads], threads
    monkeypatch.setattr(bench, "oracle_period_rate", fake)
    monkeypatch.setattr(bench, "host_cores", lambda: 16)
    cb = bench.cpu_baseline({"n_alpha": 100_000_000, "resample_every": 10})
    assert seen == [(1_000_000, 1), (8_000_000, 16)]
    assert cb["cores"] == 16 and cb["kind"] == "oracle"
    assert cb["value"] == pytest.approx(10 * 8_000_000 * 16)
    assert cb["single_thread"]["cores"] == 1
    assert cb["single_thread"]["value"] == pytest.approx(10 * 1_000_000)


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
    bench.warm_up(Sim(), None, 10, 4)
    assert calls == [("run", 10)] * 3 + [("autotune",), ("profile", True), ("run", 10)]


def test_workload_selection(bench):
    A = bench.parse(["--workload", "gauss2d_fp32_n1e8", "--strategy", "sp2"])
    wl = bench.workload(A)
    assert wl["n_alpha"] == 100_000_000 and wl["strategy"] == "sp2"
    A.particles = 1.5e7
    assert bench.workload(A)["n_alpha"] == 15_000_000
    A.workload, A.particles = "he4d_fp32_n5e7", 0
    assert bench.workload(A)["dim"] == 4
    d = bench.parse([])
    assert d.workload == "gauss2d_fp32_n1e8" and d.gpus == 1 and not d.no_secondary


def test_one_launch_period_roofline_counts_both_phases(bench):
    wl = {"precision": "fp32", "resample_every": 10, "strategy": "sp1"}
    r = bench.roofline_period(wl, ms=8.0, n=2, psteps_first=3.2e9, cand=2e8, pairs=1.2e8,
                              ceiling=5e11, clk={"sm_mhz": 2070.0}, peaks={})
    calls = 0.1 * 3.2e9 + 2e8 + 1.2e8
    assert r["achieved"] == pytest.approx(calls / 8e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 500.0)
    assert r["launch_ms"] == pytest.approx(4.0) and r["kernel"] == "k_period<fp32>"
    c0 = {"particle_steps_first": 0, "candidates": 0, "first_pairs": 0}
    c1 = {"particle_steps_first": 3.2e9, "candidates": 2e8, "first_pairs": 1.2e8}
    # the measured bytes per candidate interval scale to the launch's candidates
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PERIOD_PER_CANDIDATE["fp32"] * 1e8)
    assert bench.roofline_period(dict(wl, strategy="sp2"), 8.0, 2, 3.2e9, 2e8, 1.2e8, 5e11,
                                 {}, {})["traffic"] is None
    roof, roof2 = bench.rooflines(wl, c0, c1, (8.0, 2), (0.0, 0), 5e11, {"sm_mhz": 2070.0}, {})
    assert roof["kernel"] == "k_period<fp32>" and roof2 is None


def test_clock_record_of_a_region_shorter_than_the_first_sample(bench, tmp_path):
    """A timed region that ends before nvidia-smi's first sample gives an
    empty clock record (no median, no reasons), not a missing one; the
    rooflines then fall back to the maximum clock."""
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    c.fh = open(c.path, "w")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    c.proc = Done()
    rec = c.stop()
    assert rec["samples"] == 0 and rec["sm_mhz"] is None and rec["reasons"] == []
    r = bench.roofline({"precision": "fp32", "resample_every": 10}, 4.0, 2, 3.2e9, None, rec, {})
    assert r["peak_derived"] == pytest.approx(152 * 64 * 2070e6 / 42.0 / 1e9)
