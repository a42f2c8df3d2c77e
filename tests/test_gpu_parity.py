"""GPU parity: the CUDA path (through the C ABI) against the oracle.

FP64: the same counter-based streams and the same operation order on both
sides, so ids, event logs and integer cell counts must agree bit for bit and
positions to 1e-12 relative (the only differences allowed are the last-ulp
differences of log1p/sin/cos between CUDA and the host C library).
FP32: a different stream layout by design (geometric candidate gaps), checked in law.
"""
import numpy as np
import pytest

import workloads
from helpers import make_oracle

pytestmark = pytest.mark.gpu

REL = 1e-12


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
    # 4100 particles: 16 full blocks of 256 and a ragged tail; 100 x 64 cells:
    # three full scan tiles of 2048 and a ragged one
    base = dict(n_alpha=4100, nx=100, nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2)
    base.update(over)
    return workloads.scaled(workloads.GAUSS_2D_FP64_2E5, **base)


def sim_of(wl, capacity=None, event_log=0):
    from paper_1709_02121_gb300 import Simulation
    return Simulation(wl, capacity or 40 * wl["n_alpha"] + 4096, event_log=event_log)


def oracle_of(wl, log=False):
    o = make_oracle(wl)
    o.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    if log:
        o.enable_log()
    return o


def assert_same_particles(sim, o):
    x, k, s, w, pid = sim.particles()
    ox, ok_, ow, opid = o.particles()
    assert len(pid) == len(opid)
    a, b = np.argsort(pid, kind="stable"), np.argsort(opid, kind="stable")
    assert np.array_equal(pid[a], opid[b])
    assert np.all(np.abs(x[a] - ox[b]) <= REL * np.maximum(1.0, np.abs(ox[b])))
    assert np.all(np.abs(k[a] - ok_[b]) <= REL * np.maximum(1.0, np.abs(ok_[b])))
    assert np.all(np.sign(w[a]) == np.sign(ow[b]))
    if sim.w is not None:
        assert np.all(np.abs(w[a] - ow[b]) <= REL * np.maximum(1.0, np.abs(ow[b])))
    return x[a], k[a]


def assert_same_log(glog, olog):
    assert len(glog) == len(olog)
    kg = np.lexsort((glog["j"], glog["pid"], glog["step"]))
    ko = np.lexsort((olog["j"], olog["pid"], olog["step"]))
    g, o = glog[kg], olog[ko]
    for f in ("pid", "pid_plus", "pid_minus", "step", "j", "kill_plus", "kill_minus"):
        assert np.array_equal(g[f], o[f]), f
    for f in ("t", "xe", "kappa", "factor"):
        assert np.all(np.abs(g[f] - o[f]) <= REL * np.maximum(1.0, np.abs(o[f]))), f


def assert_same_ledger(sim, o):
    c = sim.counters()
    led = o.ledger()
    for a, b in (("events", "events"), ("kill_plus", "kill_plus"), ("kill_minus", "kill_minus"),
                 ("out_plus", "out_plus"), ("out_minus", "out_minus"),
                 ("particle_steps", "particle_steps"), ("candidates", "candidates"),
                 ("first_pairs", "first_pairs")):
        assert c[a] == led[b], (a, c[a], led[b])


# ---------------------------------------------------------------------------
def test_initial_sampling_matches_oracle():
    wl = small()
    sim, o = sim_of(wl), oracle_of(wl)
    x, k, s, w, pid = sim.particles()
    ox, ok_, ow, opid = o.particles()
    assert np.array_equal(pid, opid)
    assert np.max(np.abs(x - ox)) <= 1e-13 and np.max(np.abs(k - ok_)) <= 1e-14
    assert np.all(s == 1)


@pytest.mark.parametrize("steps", [1, 7, 13])
def test_steps_match_oracle(steps):
    wl = small(kmin=0.0, kmax=3.2, nk=32)   # narrow K: offspring get killed
    sim, o = sim_of(wl, event_log=200000), oracle_of(wl, log=True)
    sim.step(steps)
    o.step(steps)
    assert_same_particles(sim, o)
    assert_same_log(sim.event_log(), o.event_log())
    assert_same_ledger(sim, o)
    c = sim.counters()
    assert c["kill_plus"] + c["kill_minus"] > 0


def test_steps_in_pieces_equal_one_call():
    wl = small()
    a, b = sim_of(wl), sim_of(wl)
    a.step(9)
    for n in (2, 3, 4):
        b.step(n)
    xa, ka, _, _, pa = a.particles()
    xb, kb, _, _, pb = b.particles()
    ia, ib = np.argsort(pa), np.argsort(pb)
    assert np.array_equal(pa[ia], pb[ib])
    assert np.array_equal(xa[ia], xb[ib]) and np.array_equal(ka[ia], kb[ib])


def test_annihilation_and_regeneration_match_oracle():
    wl = small()
    sim, o = sim_of(wl), oracle_of(wl)
    sim.step(10)
    o.step(10)
    sim.annihilate()
    o.annihilate()
    assert np.array_equal(sim.grid_counts(), o.grid())
    assert_same_ledger(sim, o)
    # the regenerated set: ids epoch<<40 | slot, cell-major
    x, k, s, w, pid = sim.particles()
    ox, ok_, ow, opid = o.particles()
    assert np.array_equal(pid, opid)
    assert np.array_equal(x, ox) and np.array_equal(k, ok_)
    assert np.array_equal(s.astype(np.float64), ow)
    # a second resampling is a no-op on both sides
    sim.annihilate()
    o.annihilate()
    assert np.array_equal(sim.grid_counts(), o.grid())
    sim.step(5)
    o.step(5)
    assert_same_particles(sim, o)


@pytest.mark.parametrize("strategy", ["sp1", "sp2", "wp"])
def test_fused_schedule_matches_oracle(strategy):
    wl = small(strategy=strategy, resample_every=6, n_alpha=3000)
    sim, o = sim_of(wl), oracle_of(wl)
    for period in range(3):
        sim.run(6)
        o.step(6)
        o.annihilate()
        assert np.array_equal(sim.grid_counts(), o.grid()), (strategy, period)
    assert_same_ledger(sim, o)
    c = sim.counters()
    if strategy == "sp2":
        bs = o.boot_stats()
        assert [c["boot_nplus"], c["boot_nminus"]] == bs["n"].tolist()
        assert [c["boot_wplus"], c["boot_wminus"]] == bs["wfix"].astype(np.int64).tolist()
        assert [c["boot_nrplus"], c["boot_nrminus"]] == bs["nr"].tolist()
    # a run that stops between two resamplings leaves the particles in place
    sim.run(4)
    o.step(4)
    assert_same_particles(sim, o)


@pytest.mark.parametrize("n_alpha,nx,nk", [
    (20_000, 100, 64),   # about 1e5 records a period, many per cell and per warp
    (3000, 4096, 520),   # 2.1e6 cells: sparse records, runs of one
])
def test_bootstrap_binning_matches_oracle(n_alpha, nx, nk):
    """The signed bootstrap's per-cell floor counts and residual sums are
    integer sums, so the warp's run sums and atomics give the oracle's
    histogram bit for bit, with dense cells and on a grid large enough that
    every record stands alone."""
    wl = small(strategy="sp2", resample_every=6, n_alpha=n_alpha, nx=nx, nk=nk)
    sim, o = sim_of(wl), oracle_of(wl)
    for period in range(2):
        sim.run(6)
        o.step(6)
        o.annihilate()
        assert np.array_equal(sim.grid_counts(), o.grid()), period
    c = sim.counters()
    bs = o.boot_stats()
    assert [c["boot_nrplus"], c["boot_nrminus"]] == bs["nr"].tolist()


def test_fused_equals_step_plus_annihilate():
    wl = small(resample_every=5)
    a, b = sim_of(wl), sim_of(wl)
    a.run(15)
    for _ in range(3):
        b.step(5)
        b.annihilate()
    assert np.array_equal(a.grid_counts(), b.grid_counts())
    ca, cb = a.counters(), b.counters()
    for key in ("events", "kill_plus", "kill_minus", "out_plus", "out_minus", "particle_steps"):
        assert ca[key] == cb[key], key


def test_observables_match_oracle():
    wl = small()
    sim, o = sim_of(wl), oracle_of(wl)
    sim.step(6)
    o.step(6)
    # between resamplings: histogram of the particles on the fly
    dens, marg, T, live = sim.density()
    c, _ = o.histogram()
    odens, omarg, oT = o.observables(c)
    assert live == o.n
    assert np.array_equal(dens, odens) and np.array_equal(marg, omarg) and T == oT
    sim.annihilate()
    o.annihilate()
    dens, marg, T, live = sim.density()
    odens, omarg, oT = o.observables(o.grid())
    assert live == o.n and np.array_equal(dens, odens) and T == oT
    # the same read into caller-given (pinned) host buffers
    import torch
    from paper_1709_02121_gb300 import wbrw
    dh = torch.empty(wl["nx"] * wl["nk"], dtype=torch.float64).pin_memory()
    mh = torch.empty(wl["nx"], dtype=torch.float64).pin_memory()
    d2, m2, T2, live2 = wbrw.wbrw_density(sim.ctx, wl["nx"], wl["nk"], dh.numpy(), mh.numpy())
    assert np.array_equal(d2, odens) and np.array_equal(mh.numpy(), omarg)
    assert T2 == oT and live2 == live
    with pytest.raises(ValueError):
        wbrw.wbrw_density(sim.ctx, wl["nx"], wl["nk"], np.empty(3), mh.numpy())


def test_particles_leaving_the_grid_are_tallied():
    wl = small(xmin=-20.0, xmax=-12.0, nx=40, x0=-15.0)
    sim, o = sim_of(wl), oracle_of(wl)
    sim.step(8)
    o.step(8)
    sim.annihilate()
    o.annihilate()
    assert np.array_equal(sim.grid_counts(), o.grid())
    assert_same_ledger(sim, o)
    led = o.ledger()
    assert led["out_plus"] > 100


def test_empty_start():
    wl = small(n_alpha=1000)
    from paper_1709_02121_gb300 import wbrw
    sim = sim_of(wl)
    # a context with no particles at all
    ctx = wbrw.wbrw_init(sim.cfg, sim.pot, sim.bufs, 0, -15.0, 2.5, 1.5,
                         sim.stream.cuda_stream)
    wbrw.wbrw_run(ctx, 12)
    dens, marg, T, live = wbrw.wbrw_density(ctx, wl["nx"], wl["nk"])
    assert live == 0 and T == 0.0 and not dens.any()
    c = wbrw.wbrw_counters(ctx)
    assert c["particle_steps"] == 0 and c["events"] == 0
    wbrw.wbrw_destroy(ctx)


def test_capacity_overflow_is_reported():
    from paper_1709_02121_gb300 import WbrwError, wbrw
    wl = small(n_alpha=2000)
    sim = sim_of(wl, capacity=2050)
    with pytest.raises(WbrwError) as ei:
        sim.step(20)
        sim.counters()
    assert ei.value.status == wbrw.ERR_CAPACITY
    assert "capacity" in wbrw.wbrw_last_error(sim.ctx)
    with pytest.raises(WbrwError) as ei:
        sim.step(1)
    assert ei.value.status == wbrw.ERR_STATE


def test_full_size_fp64_workload_matches_oracle():
    # the 2e5-particle FP64 workload in full: 100 steps, resampling every 10,
    # run through the fused schedule the benchmark uses
    wl = workloads.GAUSS_2D_FP64_2E5
    sim = sim_of(wl, capacity=4_000_000)
    o = oracle_of(wl)
    for period in range(wl["steps"] // wl["resample_every"]):
        sim.run(wl["resample_every"])
        o.step(wl["resample_every"])
        o.annihilate()
        g, og = sim.grid_counts(), o.grid()
        if not np.array_equal(g, og):
            bad = np.argwhere(g != og)
            pytest.fail("period %d: %d cells differ, e.g. %s" % (period, len(bad), bad[:5]))
    assert_same_ledger(sim, o)
    dens, marg, T, live = sim.density()
    odens, omarg, oT = o.observables(o.grid())
    assert T == oT and live == o.n


def test_runs_are_deterministic():
    wl = small(precision="fp32", n_alpha=200000, resample_every=5)
    a, b = sim_of(wl, capacity=3_000_000), sim_of(wl, capacity=3_000_000)
    a.run(20)
    b.run(20)
    assert np.array_equal(a.grid_counts(), b.grid_counts())
    assert a.counters()["events"] == b.counters()["events"]


def test_checkpoint_restore_is_bit_identical():
    wl = small(resample_every=5)
    a, b = sim_of(wl), sim_of(wl)
    a.run(10)
    grid, step, epoch = a.checkpoint()
    assert step == 10 and epoch == 2
    a.run(10)
    b.restore(grid, step, epoch)      # host memory
    b.run(10)
    assert np.array_equal(a.grid_counts(), b.grid_counts())
    # from device memory, then the particles themselves
    import torch
    c = sim_of(wl)
    c.restore(torch.from_numpy(grid.copy()).cuda(), step, epoch)
    c.run(3)
    a2 = sim_of(wl)
    a2.run(13)
    xa, ka, _, _, pa = a2.particles()
    xc, kc, _, _, pc = c.particles()
    ia, ic = np.argsort(pa), np.argsort(pc)
    assert np.array_equal(pa[ia], pc[ic]) and np.array_equal(xa[ia], xc[ic])
    # a checkpoint between resamplings is refused
    from paper_1709_02121_gb300 import WbrwError
    with pytest.raises(WbrwError):
        c.checkpoint()
