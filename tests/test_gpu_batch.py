"""GPU parity of batches: many independent problems in the same launches.

Instance i of a batch is the run the oracle makes with that instance's
potential, wavepacket, rate and N_alpha and with the instance salt i in its
particle labels.  FP64: ids, integer cell counts and ledgers bit for bit,
positions to 1e-12 relative, per instance.  Both precisions: an instance does
not depend on the others (a batch and its prefix agree bit for bit), and
instance 0 is the plain run.
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


# 100 x 64 cells per instance: three full scan tiles and a ragged one each,
# so instance boundaries fall inside scan tiles
BASE = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, nx=100, nk=64, xmin=-25.0, xmax=25.0,
                        kmin=-3.2, kmax=3.2, resample_every=5)

# uneven problems: different barriers, packets and sizes, one of them empty,
# one with a rate above the majorant
INSTANCES = [
    dict(H=1.0, w=1.0, x0=-8.0, sigma_x=2.0, k0=1.5, n_init=4100, n_alpha=4100),
    dict(H=0.5, w=1.7, x0=-6.0, sigma_x=1.5, k0=2.2, n_init=700, n_alpha=700),
    dict(H=2.0, w=0.6, x0=-4.0, sigma_x=1.0, k0=1.1, n_init=2500, n_alpha=2500),
    dict(H=1.3, w=0.9, x0=-5.0, sigma_x=1.2, k0=1.8, n_init=0, n_alpha=100),
    dict(H=-0.8, w=1.2, x0=-7.0, sigma_x=1.8, k0=1.3, n_init=1500, n_alpha=1500,
         gamma0=1.4),
]


def batch_of(wl, insts, capacity=400_000):
    from paper_1709_02121_gb300 import Batch
    return Batch(wl, insts, capacity)


def oracle_of(wl, i, inst):
    o = make_oracle(wl, H=inst["H"], w=inst["w"], n_alpha=inst["n_alpha"],
                    gamma0=inst.get("gamma0", 0.0), instance=i)
    o.init_gauss(inst["n_init"], inst["x0"], inst["sigma_x"], inst["k0"])
    return o


def split(arrs, inst, i):
    m = inst == i
    return [a[m] for a in arrs]


def test_initial_sampling_per_instance():
    b = batch_of(BASE, INSTANCES)
    x, k, s, w, pid, inst = b.particles()
    assert len(x) == sum(v["n_init"] for v in INSTANCES)
    for i, v in enumerate(INSTANCES):
        xi, ki, pi = split((x, k, pid), inst, i)
        o = oracle_of(BASE, i, v)
        ox, ok_, _, opid = o.particles()
        assert np.array_equal(pi, opid)
        assert np.all(np.abs(xi - ox) <= REL * np.maximum(1.0, np.abs(ox)))
        assert np.all(np.abs(ki - ok_) <= REL * np.maximum(1.0, np.abs(ok_)))


def test_steps_match_oracle_per_instance():
    b = batch_of(BASE, INSTANCES)
    b.step(7)
    x, k, s, w, pid, inst = b.particles()
    for i, v in enumerate(INSTANCES):
        xi, ki, si, pi = split((x, k, s, pid), inst, i)
        o = oracle_of(BASE, i, v)
        o.step(7)
        ox, ok_, ow, opid = o.particles()
        assert len(pi) == len(opid), i
        a, c = np.argsort(pi, kind="stable"), np.argsort(opid, kind="stable")
        assert np.array_equal(pi[a], opid[c]), i
        assert np.all(np.abs(xi[a] - ox[c]) <= REL * np.maximum(1.0, np.abs(ox[c]))), i
        assert np.all(np.abs(ki[a] - ok_[c]) <= REL * np.maximum(1.0, np.abs(ok_[c]))), i
        assert np.array_equal(si[a].astype(np.float64), ow[c]), i
        _, _, _, live = b.density(i)
        assert live == o.n, i


def test_fused_schedule_matches_oracle_per_instance():
    b = batch_of(BASE, INSTANCES)
    ors = [oracle_of(BASE, i, v) for i, v in enumerate(INSTANCES)]
    for period in range(3):
        b.run(5)
        g = b.grid_counts()
        for i, o in enumerate(ors):
            o.step(5)
            o.annihilate()
            assert np.array_equal(g[i], o.grid()), (period, i)
    # ledgers are sums over instances
    c = b.counters()
    leds = [o.ledger() for o in ors]
    for key in ("events", "kill_plus", "kill_minus", "out_plus", "out_minus", "particle_steps",
                "candidates", "first_pairs"):
        assert c[key] == sum(led[key] for led in leds), key
    # observables per instance, and all transmissions at once
    T_all = b.transmissions()
    for i, o in enumerate(ors):
        dens, marg, T, live = b.density(i)
        odens, omarg, oT = o.observables(o.grid())
        assert np.array_equal(dens, odens) and np.array_equal(marg, omarg), i
        assert T == oT and T_all[i] == oT and live == o.n, i
    assert T_all[3] == 0.0
    # regenerated particles carry (epoch << 40) | (instance << 32) | j
    b.run(2)
    x, k, s, w, pid, inst = b.particles()
    for i, o in enumerate(ors):
        o.step(2)
        pi, xi = split((pid, x), inst, i)
        ox, _, _, opid = o.particles()
        a, c2 = np.argsort(pi, kind="stable"), np.argsort(opid, kind="stable")
        assert np.array_equal(pi[a], opid[c2]), i
        assert np.all(np.abs(xi[a] - ox[c2]) <= REL * np.maximum(1.0, np.abs(ox[c2]))), i


@pytest.mark.parametrize("strategy", ["sp2", "wp"])
def test_weighted_strategies_match_oracle_per_instance(strategy):
    """sp2 bootstraps each instance on its own (Alg. 2 per instance and side,
    its shares from the instance's N^s and W^s) and wp rounds each instance's
    weighted histogram; the residual draws and the roundings carry the
    instance salt.  FP64: every instance's histogram equals the salted
    oracle's after each period, the sp2 filter's totals are the sums of the
    instances' (the empty instance and the one with H < 0 included)."""
    wl = workloads.scaled(BASE, strategy=strategy)
    b = batch_of(wl, INSTANCES)
    ors = [oracle_of(wl, i, v) for i, v in enumerate(INSTANCES)]
    for period in range(3):
        b.run(5)
        g = b.grid_counts()
        for i, o in enumerate(ors):
            o.step(5)
            o.annihilate()
            assert np.array_equal(g[i], o.grid()), (period, i)
        if strategy == "sp2":
            c = b.counters()
            st = [o.boot_stats() for o in ors]
            for key, name, side in (("boot_nplus", "n", 0), ("boot_nminus", "n", 1),
                                    ("boot_nrplus", "nr", 0), ("boot_nrminus", "nr", 1),
                                    ("boot_wplus", "wfix", 0), ("boot_wminus", "wfix", 1)):
                assert c[key] == sum(int(s_[name][side]) for s_ in st), (period, key)
    c = b.counters()
    leds = [o.ledger() for o in ors]
    for key in ("events", "kill_plus", "kill_minus", "out_plus", "out_minus", "particle_steps"):
        assert c[key] == sum(led[key] for led in leds), key
    b.run(2)
    x, k, s, w, pid, inst = b.particles()
    for i, o in enumerate(ors):
        o.step(2)
        pi, xi, wi = split((pid, x, w), inst, i)
        ox, _, ow, opid = o.particles()
        a, c2 = np.argsort(pi, kind="stable"), np.argsort(opid, kind="stable")
        assert np.array_equal(pi[a], opid[c2]), i
        assert np.all(np.abs(xi[a] - ox[c2]) <= REL * np.maximum(1.0, np.abs(ox[c2]))), i
        assert np.all(np.abs(wi[a] - ow[c2]) <= REL * np.maximum(1.0, np.abs(ow[c2]))), i


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("strategy", ["sp1", "sp2", "wp"])
def test_instances_do_not_interact(precision, strategy):
    wl = workloads.scaled(BASE, precision=precision, strategy=strategy)
    full = batch_of(wl, INSTANCES)
    prefix = batch_of(wl, INSTANCES[:2])
    full.run(10)
    prefix.run(10)
    gf, gp = full.grid_counts(), prefix.grid_counts()
    assert np.array_equal(gf[:2], gp)
    # instance 0 of a batch is the plain run
    from paper_1709_02121_gb300 import Simulation
    v = INSTANCES[0]
    plain = Simulation(workloads.scaled(wl, H=v["H"], w=v["w"], x0=v["x0"],
                                        sigma_x=v["sigma_x"], k0=v["k0"],
                                        n_alpha=v["n_alpha"]), 400_000)
    plain.run(10)
    assert np.array_equal(gf[0], plain.grid_counts())


def test_batch_checkpoint_restore_is_bit_identical():
    a, b = batch_of(BASE, INSTANCES), batch_of(BASE, INSTANCES)
    a.run(5)
    grid, step, epoch = a.checkpoint()
    assert grid.shape == (len(INSTANCES), BASE["nx"], BASE["nk"])
    a.run(10)
    b.restore(grid, step, epoch)
    b.run(10)
    assert np.array_equal(a.grid_counts(), b.grid_counts())


def test_batch_arguments_are_checked():
    from paper_1709_02121_gb300 import WbrwError
    with pytest.raises(WbrwError):   # more initial particles than slots
        batch_of(BASE, INSTANCES, capacity=5000)
    with pytest.raises(WbrwError):   # a rate below the majorant C/2
        batch_of(BASE, [dict(INSTANCES[0], gamma0=0.3)])
    with pytest.raises((WbrwError, ValueError)):   # too many instances
        batch_of(BASE, [dict(INSTANCES[1], n_init=1)] * 257)
