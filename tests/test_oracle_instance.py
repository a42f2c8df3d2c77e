"""Oracle: the instance salt that makes the runs of a batch independent.

A batch runs several problems side by side with one seed; instance i of
the batch labels its particles (i << 32) | index at start and
(epoch << 40) | (i << 32) | j after the regeneration of Alg. 3, so that
no two instances share a random stream.  Pins: the label layout, the
instance-0 run being the plain run, and a salted run differing from it
while keeping the Gaussian initial statistics of Sec. 5 (x ~ N(x0, sx^2)).
"""
import numpy as np
import pytest

import oracle
from helpers import make_oracle
import workloads
from workloads import COLLISION_2D


def _run(instance, n=4000, steps=0):
    o = make_oracle(COLLISION_2D, n_alpha=n, instance=instance)
    o.init_gauss(n, COLLISION_2D["x0"], COLLISION_2D["sigma_x"], COLLISION_2D["k0"])
    if steps:
        o.step(steps)
    return o


def test_initial_labels_carry_the_instance():
    o = _run(7)
    _, _, w, pid = o.particles()
    assert np.array_equal(pid, (np.uint64(7) << np.uint64(32)) + np.arange(len(pid), dtype=np.uint64))
    assert np.all(w == 1.0)


def test_instance_zero_is_the_plain_run():
    a = make_oracle(COLLISION_2D, n_alpha=3000)
    a.init_gauss(3000, COLLISION_2D["x0"], COLLISION_2D["sigma_x"], COLLISION_2D["k0"])
    a.step(3)
    b = _run(0, n=3000, steps=3)
    for u, v in zip(a.particles(), b.particles()):
        assert np.array_equal(u, v)


def test_salted_run_differs_but_keeps_the_initial_law():
    x0, sx = COLLISION_2D["x0"], COLLISION_2D["sigma_x"]
    xa = _run(0, n=20000).particles()[0]
    xb = _run(3, n=20000).particles()[0]
    assert not np.array_equal(xa, xb)
    for x in (xa, xb):
        # mean within 5 standard errors, variance within 5 standard errors
        assert abs(x.mean() - x0) < 5 * sx / np.sqrt(len(x))
        assert abs(x.var() / sx**2 - 1.0) < 5 * np.sqrt(2.0 / len(x))


def test_regenerated_labels_carry_epoch_and_instance():
    o = _run(200, n=3000, steps=2)
    o.annihilate()
    _, _, _, pid = o.particles()
    ep = pid >> np.uint64(40)
    inst = (pid >> np.uint64(32)) & np.uint64(0xFF)
    j = pid & np.uint64(0xFFFFFFFF)
    assert np.all(ep == o.epoch) and o.epoch >= 1
    assert np.all(inst == 200)
    assert np.array_equal(j, np.arange(len(pid), dtype=np.uint64))


@pytest.mark.parametrize("bad", [-1, 256])
def test_out_of_range_instance_is_rejected(bad):
    with pytest.raises(ValueError):
        make_oracle(COLLISION_2D, instance=bad)


# ---------------------------------------------------------------------------
# The resampling streams of a salted run: sp2's residual draws and roundings
# and wp's roundings are counted (instance << 32) | d and
# (instance << 32) | nu, so that the instances of a batch (salt 0: the plain
# run) draw from separate streams.
# ---------------------------------------------------------------------------
GRID3 = dict(nx=3, nk=1, xmin=0.0, xmax=3.0, kmin=0.0, kmax=1.0)
STEP_BOOT, STEP_ROUND = 0xFFFFFFFD, 0xFFFFFFFC


def _philox(seed, ctr):
    return oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])


@pytest.mark.parametrize("strategy", ["sp2", "wp"])
def test_instance_zero_resamples_as_the_plain_run(strategy):
    wl = dict(COLLISION_2D, strategy=strategy)
    a = make_oracle(wl, n_alpha=3000)
    b = make_oracle(wl, n_alpha=3000, instance=0)
    for o in (a, b):
        o.init_gauss(3000, COLLISION_2D["x0"], COLLISION_2D["sigma_x"], COLLISION_2D["k0"])
        o.step(4)
        o.annihilate()
    assert np.array_equal(a.grid(), b.grid())
    if strategy == "sp2":
        for u, v in zip(a.boot_counts(), b.boot_counts()):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("instance", [0, 5, 255])
def test_salted_bootstrap_draws_and_rounding(instance):
    """Three cells holding positive weights 1/2, 1/4, 1/4: N = 3, W = 1, shares
    q = (3/2, 3/4, 3/4), kept floor(q) = (1, 0, 0), residuals (1/2, 3/4, 3/4)
    with prefix (1/2, 5/4, 2) and N_r = 2 draws (Alg. 2).  Draw d takes the 64
    bits r of Philox at ((b << 32) | d, BOOT, epoch << 1) and picks the first
    cell whose prefix exceeds floor(r R / 2^64); then m_nu = (W/N) n~_nu is
    rounded by the uniform of ((b << 32) | nu, ROUND, epoch) (Alg. 3)."""
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, strategy="sp2", n_alpha=3, **GRID3)
    o = make_oracle(wl, instance=instance)
    o.set_particles(np.array([0.5, 1.5, 2.5]), np.full(3, 0.5), np.array([0.5, 0.25, 0.25]),
                    np.arange(3, dtype=np.uint64))
    o.annihilate()
    e, seed = o.epoch, wl["seed"]
    R = 1 << 33                                        # 2 in Q0.32
    prefix = [1 << 31, 5 << 30, 1 << 33]
    n = [1, 0, 0]
    for d in range(2):
        h = _philox(seed, [d, instance, STEP_BOOT, e << 1])
        U = (((int(h[1]) << 32) | int(h[0])) * R) >> 64
        n[next(i for i, p in enumerate(prefix) if p > U)] += 1
    plus, minus = o.boot_counts()
    assert plus[:, 0].tolist() == n and not minus.any()
    st = o.boot_stats()
    assert st["n"].tolist() == [3, 0] and st["keep"].tolist() == [1, 0]
    assert st["nr"].tolist() == [2, 0]
    amp = 1.0 / 3.0                                    # (W 2^-31) / N
    expect = []
    for nu in range(3):
        m = n[nu] * amp
        h = _philox(seed, [nu, instance, STEP_ROUND, e])
        fl = np.floor(m)
        expect.append(int(fl) + (1 if oracle.u53(h[0], h[1]) < m - fl else 0))
    assert o.grid()[:, 0].tolist() == expect


@pytest.mark.parametrize("instance", [0, 7])
def test_salted_wp_rounding(instance):
    """The weighted histogram of Eq. piecewise_constant_function (weights in
    units of 2^-31) rounded by Alg. 3 with the uniform of
    ((b << 32) | nu, ROUND, epoch)."""
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, strategy="wp", n_alpha=4, **GRID3)
    o = make_oracle(wl, instance=instance)
    w = np.array([0.3, -0.45, 0.8, 0.6])
    cells = np.array([0, 1, 2, 2])
    o.set_particles(cells + 0.5, np.full(4, 0.5), w, np.arange(4, dtype=np.uint64))
    o.annihilate()
    e, seed = o.epoch, wl["seed"]
    ws = np.zeros(3, np.int64)
    np.add.at(ws, cells, np.rint(w * 2.0 ** 31).astype(np.int64))
    expect = []
    for nu in range(3):
        m = ws[nu] * 2.0 ** -31
        am = abs(m)
        h = _philox(seed, [nu, instance, STEP_ROUND, e])
        cnt = int(np.floor(am)) + (1 if oracle.u53(h[0], h[1]) < am - np.floor(am) else 0)
        expect.append(-cnt if m < 0 else cnt)
    assert o.grid()[:, 0].tolist() == expect
