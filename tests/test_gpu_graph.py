"""CUDA-graph replay of resampling periods (wbrw_graph).

A replayed period must be bit for bit the period launched kernel by kernel:
the kernels read the period's first interval and id base from device memory
and the graph advances them, so every replay continues the run.  Checked
against the eager path for plain runs and batches, across a mix of graph
periods and eager operations (steps, annihilation, restore), and against the
oracle in FP64.
"""
import numpy as np
import pytest

import workloads
from helpers import make_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def small(**over):
    base = dict(n_alpha=4100, nx=100, nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2,
                resample_every=5)
    base.update(over)
    return workloads.scaled(workloads.GAUSS_2D_FP64_2E5, **base)


def sim(wl, graph, gpu, capacity=400_000, event_log=0):
    from paper_1709_02121_gb300 import Simulation
    s = Simulation(wl, capacity, event_log=event_log, stream=gpu.cuda.Stream())
    if graph:
        s.graph(True)
    return s


KEYS = ("events", "kill_plus", "kill_minus", "out_plus", "out_minus", "particle_steps",
        "particle_steps_first", "live", "step", "epoch", "candidates", "first_pairs")


@pytest.mark.parametrize("strategy", ["sp1", "sp2", "wp"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_replayed_periods_equal_eager_periods(gpu, precision, strategy):
    wl = small(precision=precision, strategy=strategy)
    a, b = sim(wl, False, gpu), sim(wl, True, gpu)
    for period in range(6):
        a.run(5)
        b.run(5)
        assert np.array_equal(a.grid_counts(), b.grid_counts()), period
    ca, cb = a.counters(), b.counters()
    keys = KEYS + (("boot_nplus", "boot_nminus", "boot_nrplus", "boot_nrminus", "boot_wplus",
                    "boot_wminus") if strategy == "sp2" else ())
    for k in keys:
        assert ca[k] == cb[k], k
    # the same kernels, plus one period-state advance per replay (periods 2-6)
    # and one initial period-state write
    assert cb["launches"] - ca["launches"] == 5 + 1


@pytest.mark.parametrize("strategy", ["sp1", "sp2", "wp"])
def test_replays_match_the_oracle_fp64(gpu, strategy):
    wl = small(n_alpha=3000, strategy=strategy)
    s = sim(wl, True, gpu)
    o = make_oracle(wl)
    o.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    for period in range(4):
        s.run(5)
        o.step(5)
        o.annihilate()
        assert np.array_equal(s.grid_counts(), o.grid()), period


def test_graph_periods_mixed_with_eager_operations(gpu):
    wl = small()

    def script(s):
        s.run(10)            # the first period from the initial particles, then a replay
        s.step(3)            # particles into the arrays, eager
        s.run(2)             # to the boundary: eager (the source is the arrays)
        s.run(12)            # two replays and two steps
        s.run(3)             # to the next boundary
        grid, step, epoch = s.checkpoint()
        s.run(5)
        s.restore(grid, step, epoch)   # back one period, the graph state follows
        s.run(10)
        return s.grid_counts(), s.counters()

    ga, ca = script(sim(wl, False, gpu))
    gb, cb = script(sim(wl, True, gpu))
    assert np.array_equal(ga, gb)
    for k in ("events", "particle_steps", "live", "step", "epoch"):
        assert ca[k] == cb[k], k


def test_batch_replays_equal_eager(gpu):
    from paper_1709_02121_gb300 import Batch
    wl = workloads.scaled(small(), precision="fp32")
    insts = [dict(H=1.0, w=1.0, x0=-8.0, sigma_x=2.0, k0=1.5, n_init=3000, n_alpha=3000),
             dict(H=1.8, w=0.7, x0=-5.0, sigma_x=1.5, k0=2.0, n_init=500, n_alpha=500),
             dict(H=0.6, w=1.5, x0=-6.0, sigma_x=1.0, k0=1.2, n_init=1200, n_alpha=1200)]
    a = Batch(wl, insts, 200_000, stream=gpu.cuda.Stream())
    b = Batch(wl, insts, 200_000, stream=gpu.cuda.Stream())
    b.graph(True)
    for _ in range(5):
        a.run(5)
        b.run(5)
    assert np.array_equal(a.grid_counts(), b.grid_counts())
    assert np.array_equal(a.transmissions(), b.transmissions())


def test_profiling_sees_every_replayed_first_wave(gpu):
    from paper_1709_02121_gb300 import wbrw
    s = sim(small(precision="fp32", n_alpha=50_000), True, gpu, capacity=1_000_000)
    s.run(10)
    wbrw.wbrw_profile(s.ctx, True)
    s.run(20)
    ms, n = wbrw.wbrw_profile_read(s.ctx)
    assert n == 4 and ms > 0


@pytest.mark.parametrize("graphs", [False, True])
def test_profiling_sees_every_event_kernel(gpu, graphs):
    # an event log selects the general kernels, which launch the event kernel
    # once per round (the lean ones run a whole period in one launch)
    from paper_1709_02121_gb300 import wbrw
    s = sim(small(precision="fp32", n_alpha=50_000), graphs, gpu, capacity=1_000_000,
            event_log=1 << 16)
    s.run(10)
    wbrw.wbrw_profile(s.ctx, True)
    s.run(20)
    ms_f, n_f = wbrw.wbrw_profile_read(s.ctx)
    ms_e, n_e = wbrw.wbrw_profile_read_events(s.ctx)
    # one event-kernel launch per round: 4 periods of 5 rounds
    assert n_f == 4 and n_e == 20 and ms_e > 0
    assert wbrw.wbrw_profile_read_events(s.ctx) == (0.0, 0)
    # off again: replays point the records back at their placeholders
    wbrw.wbrw_profile(s.ctx, False)
    s.run(10)
    assert wbrw.wbrw_profile_read_events(s.ctx)[1] == 0
    wbrw.wbrw_profile(s.ctx, True)
    s.run(5)
    assert wbrw.wbrw_profile_read_events(s.ctx)[1] == 5


@pytest.mark.parametrize("graphs", [False, True])
def test_profiling_sees_every_one_launch_period(gpu, graphs):
    """The lean kernels run a regenerating period in one launch, which the
    first-wave records time; no event-kernel launch is left to time."""
    from paper_1709_02121_gb300 import wbrw
    s = sim(small(precision="fp32", n_alpha=50_000), graphs, gpu, capacity=1_000_000)
    s.run(10)
    wbrw.wbrw_profile(s.ctx, True)
    s.run(20)
    ms_f, n_f = wbrw.wbrw_profile_read(s.ctx)
    ms_e, n_e = wbrw.wbrw_profile_read_events(s.ctx)
    assert n_f == 4 and ms_f > 0 and n_e == 0


def test_graphs_need_a_created_stream(gpu):
    from paper_1709_02121_gb300 import Simulation, WbrwError, wbrw
    s = Simulation(small(), 100_000, stream=gpu.cuda.default_stream())
    with pytest.raises(WbrwError) as ei:
        s.graph(True)
    assert ei.value.status == wbrw.ERR_ARG


@pytest.mark.parametrize("graphs", [False, True])
def test_profiling_changes_no_result(gpu, graphs):
    """The profiling records sit on a side stream (a side branch of a
    captured period): switching them on and off, which captures the period
    again, leaves every count and cell bit-identical."""
    from paper_1709_02121_gb300 import wbrw
    wl = small(precision="fp32", n_alpha=50_000)
    a = sim(wl, graphs, gpu, capacity=1_000_000)
    b = sim(wl, graphs, gpu, capacity=1_000_000)
    for i in range(6):
        wbrw.wbrw_profile(b.ctx, i % 2 == 1)
        a.run(5)
        b.run(5)
    ca, cb = a.counters(), b.counters()
    for key in KEYS:
        assert ca[key] == cb[key], key
    assert np.array_equal(a.grid_counts(), b.grid_counts())

