"""The oracle's threaded mode gives the serial results bit for bit.

Every draw is keyed by (particle id, interval, draw), so the order in which
particles are processed cannot change a result.  The threaded mode cuts each
interval's particle list into contiguous chunks, keeps each chunk's outputs
apart and joins them in chunk order; binning adds integers; regeneration
places each cell's particles at their position in cell order.  These tests
run the same workload with 1, 3 and 7 chunks (7 does not divide the particle
counts) and compare particles, ids, grids, ledgers and event logs.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import make_oracle


def _run(wl, threads, periods, log=False):
    o = make_oracle(wl, threads=threads)
    if log:
        o.enable_log()
    o.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    grids = []
    for _ in range(periods):
        o.step(wl["resample_every"])
        o.annihilate()
        grids.append(o.grid().copy())
    o.step(3)
    return o, grids


@pytest.mark.parametrize("strategy", ["sp1", "sp2"])
def test_threads_do_not_change_any_result(strategy):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=20_011, strategy=strategy,
                          resample_every=5)
    ref, gref = _run(wl, 1, 3, log=True)
    for t in (3, 7):
        o, g = _run(wl, t, 3, log=True)
        assert o.threads == t
        for a, b in zip(gref, g):
            assert np.array_equal(a, b)
        for a, b in zip(ref.particles(), o.particles()):
            assert np.array_equal(a, b)
        assert ref.ledger() == o.ledger()
        assert np.array_equal(ref.event_log(), o.event_log())
        if strategy == "sp2":
            for k in ("n", "keep", "nr", "wfix"):
                assert np.array_equal(ref.boot_stats()[k], o.boot_stats()[k])


def test_threads_with_tangents_keep_particles_and_dgrid():
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=6_007, resample_every=4,
                          tangent=True, tquantum=0.5)
    ref, _ = _run(wl, 1, 2)
    o, _ = _run(wl, 5, 2)
    for a, b in zip(ref.particles(), o.particles()):
        assert np.array_equal(a, b)
    for a, b in zip(ref.tangent(), o.tangent()):
        assert np.array_equal(a, b)


def test_thread_count_is_reported():
    assert oracle.max_threads() >= 1
    with pytest.raises(ValueError):
        oracle.Oracle(threads=0)
