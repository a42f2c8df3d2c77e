"""Launch-shape tuning and the autotuner.

The shape (resident blocks per SM, which also sets the queue segmentation,
and the number of lockstep event passes before the recursive drain) must not
change any result: random numbers are keyed by particle and interval and
every count is an integer sum.  The autotuner must leave the run exactly as
it found it.
"""
import numpy as np
import pytest

import workloads

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
    # narrow K: offspring get killed; H = 2: several events per interval, so
    # deferred segments reach the deepest levels
    base = dict(n_alpha=6000, nx=100, nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2,
                resample_every=5, H=2.0, w=0.6)
    base.update(over)
    return workloads.scaled(workloads.GAUSS_2D_FP64_2E5, **base)


def sim(wl, event_log=0):
    from paper_1709_02121_gb300 import Simulation
    return Simulation(wl, 600_000, event_log=event_log)


SHAPES = [(1, 0), (2, 1), (3, 3), (1, 6), (3, 6), (2, 0)]
# FP32 runs with one instance, the static potential and no event log run
# kernels built for four blocks per SM
SHAPES_LEAN = SHAPES + [(4, 0), (4, 3)]
KEYS = ("events", "kill_plus", "kill_minus", "out_plus", "out_minus", "particle_steps", "live")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_results_do_not_depend_on_the_shape(precision):
    wl = small(precision=precision)
    ref = sim(wl)
    ref.run(15)
    ref.step(4)
    xr, kr, _, _, pr = ref.particles()
    order = np.argsort(pr)
    for b, p in (SHAPES_LEAN if precision == "fp32" else SHAPES):
        s = sim(wl)
        assert s.tuning(b, p) == (b, p)
        s.run(15)
        assert np.array_equal(s.grid_counts(), ref.grid_counts()), (b, p)
        s.step(4)
        x, k, _, _, pid = s.particles()
        o = np.argsort(pid)
        assert np.array_equal(pid[o], pr[order]), (b, p)
        assert np.array_equal(x[o], xr[order]) and np.array_equal(k[o], kr[order]), (b, p)
        cs, cr = s.counters(), ref.counters()
        for key in KEYS:
            assert cs[key] == cr[key], (b, p, key)


def test_autotune_leaves_the_run_unchanged():
    wl = small(precision="fp32", n_alpha=20000)
    a, b = sim(wl, event_log=100000), sim(wl, event_log=100000)
    a.run(5)
    b.run(5)
    log_len = b.counters()["log_len"]
    (bps, passes), table = b.autotune(trials=1)
    # the event log selects the general kernels: three blocks per SM at most
    assert table.shape == (4, 7) and np.all(table[:3] > 0) and np.all(table[3] < 0)
    assert table[bps - 1, passes] == table[:3].min()
    assert b.tuning() == (bps, passes)
    assert b.counters()["log_len"] == log_len
    a.run(10)
    b.run(10)
    assert np.array_equal(a.grid_counts(), b.grid_counts())
    ca, cb = a.counters(), b.counters()
    for key in KEYS + ("step", "epoch", "log_len"):
        assert ca[key] == cb[key], key


def test_autotune_of_the_lean_kernels_leaves_the_run_unchanged():
    wl = small(precision="fp32", n_alpha=20000)
    a, b = sim(wl), sim(wl)
    a.run(5)
    b.run(5)
    (bps, passes), table = b.autotune(trials=1)
    # deferred segments are finished inside the event kernel: only
    # event_passes = 0 is timed
    assert table.shape == (4, 7) and np.all(table[:, 0] > 0) and np.all(table[:, 1:] < 0)
    assert passes == 0 and table[bps - 1, 0] == table[:, 0].min()
    assert b.tuning() == (bps, passes)
    a.run(10)
    b.run(10)
    assert np.array_equal(a.grid_counts(), b.grid_counts())
    ca, cb = a.counters(), b.counters()
    for key in KEYS + ("step", "epoch"):
        assert ca[key] == cb[key], key


def test_tuning_arguments_are_checked():
    from paper_1709_02121_gb300 import WbrwError, wbrw
    s = sim(small())
    for bad in ((0, 3), (4, 3), (3, -1), (3, 7)):
        with pytest.raises(WbrwError) as ei:
            s.tuning(*bad)
        assert ei.value.status == wbrw.ERR_ARG
    s.step(2)
    with pytest.raises(WbrwError) as ei:     # not right after a resampling
        s.autotune()
    assert ei.value.status == wbrw.ERR_STATE
    lean = sim(small(precision="fp32"))       # built for four blocks per SM
    assert lean.tuning() == (4, 3)
    assert lean.tuning(4, 0) == (4, 0)
    for bad in ((5, 0), (0, 0)):
        with pytest.raises(WbrwError) as ei:
            lean.tuning(*bad)
        assert ei.value.status == wbrw.ERR_ARG
