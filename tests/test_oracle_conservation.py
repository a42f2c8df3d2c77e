"""Conservation and growth pins: the net signed count under pair branching,
annihilation and regeneration (Alg. 1 item 5, Eq. signed_histogram, Alg. 3),
and the growth of the particle number (Theorem 1)."""
import numpy as np

import workloads
from helpers import make_oracle, net_sign


def test_net_count_ledger_every_step(oracle_mod):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=3000,
                          kmin=0.6, kmax=2.4, nk=36)  # narrow K: many kills
    o = make_oracle(wl)
    o.init_gauss(3000, wl["x0"], wl["sigma_x"], wl["k0"])
    net = 3000
    prev = o.ledger()
    for _ in range(12):
        o.step(1)
        led = o.ledger()
        dk = (led["kill_plus"] - prev["kill_plus"]) - (led["kill_minus"] - prev["kill_minus"])
        _, _, w, _ = o.particles()
        assert net_sign(w) == net - dk
        net -= dk
        prev = led
    assert led["kill_plus"] + led["kill_minus"] > 0


def test_annihilation_conserves_in_grid_net_count(oracle_mod):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=5000,
                          nx=40, nk=32, xmin=-22.0, xmax=-2.0, kmin=0.0, kmax=3.2)
    o = make_oracle(wl)
    o.init_gauss(5000, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(10)
    x, k, w, _ = o.particles()
    before = o.ledger()
    counts, _ = o.histogram()
    o.annihilate()
    g = o.grid()
    assert np.array_equal(g, counts)
    led = o.ledger()
    out = (led["out_plus"] - before["out_plus"]) - (led["out_minus"] - before["out_minus"])
    assert g.sum() == net_sign(w) - out
    assert o.n == np.abs(g).sum()
    _, _, w2, pid2 = o.particles()
    assert net_sign(w2) == g.sum()
    assert np.all(pid2 >> np.uint64(40) == 1)   # epoch 1 ids, slots in order
    assert np.array_equal(pid2 & np.uint64((1 << 40) - 1), np.arange(o.n, dtype=np.uint64))
    # a second resampling with no step in between changes nothing
    o.annihilate()
    assert o.epoch == 1 and np.array_equal(o.grid(), g)


def test_rebin_of_regeneration_is_identity(oracle_mod):
    # a random signed grid, cells of awkward width (0.1 is not binary)
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=1000,
                          nx=50, nk=40, xmin=-2.5, xmax=2.5, kmin=-0.3, kmax=3.7)
    o = make_oracle(wl)
    rng = np.random.default_rng(3)
    g = rng.integers(-9, 10, size=(50, 40)).astype(np.int32)
    for epoch in (1, 2, 77):
        o.set_grid(g, epoch)
        o.regenerate()
        c, _ = o.histogram()
        assert np.array_equal(c, g)
        x, k, w, pid = o.particles()
        assert np.all(x >= -2.5) and np.all(x < 2.5)


def test_regeneration_is_uniform_inside_cells(oracle_mod):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=1000,
                          nx=2, nk=1, xmin=0.0, xmax=1.0, kmin=0.0, kmax=1.0)
    o = make_oracle(wl)
    o.set_grid(np.array([[20000], [-20000]], np.int32), 1)
    o.regenerate()
    x, k, w, _ = o.particles()
    left = x < 0.5
    assert np.all(w[left] == 1) and np.all(w[~left] == -1)
    from scipy import stats
    assert stats.kstest(x[left] / 0.5, "uniform").pvalue > 1e-3
    assert stats.kstest(k, "uniform").pvalue > 1e-3


def test_growth_bound_and_far_field_rate(oracle_mod):
    # Theorem 1: E Z_t <= exp(2 xi_check t) (M = 1); far from the barrier the
    # particle number grows as exp(2 xi t) with xi = 2|H|/(pi hbar)
    ratios = []
    t = 1.0
    for seed in range(6):
        wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=4000,
                              seed=seed, x0=-30.0, sigma_x=1.0)
        o = make_oracle(wl)
        o.init_gauss(4000, wl["x0"], wl["sigma_x"], wl["k0"])
        o.step(10)
        ratios.append(o.n / 4000)
    ratios = np.array(ratios)
    expect = np.exp(2 * (2 / np.pi) * t)
    se = ratios.std(ddof=1) / np.sqrt(len(ratios))
    assert abs(ratios.mean() - expect) < 4.5 * se + 0.01
    assert ratios.mean() <= expect * 1.02
