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
