"""Pins of the oracle's observables (Eq. estimator) against the particle
estimator they stand for.

The estimator of an observable A is (1/N_alpha) sum_i s_i A(x_i, k_i).  With
A the indicator of a cell divided by its measure dx dk it is the histogram
density; with A the indicator of a column divided by dx, the x-marginal; with
A = 1{x > 0}, the transmission.  A histogram only knows which cell holds a
particle, so the transmission of a histogram counts whole cells: those whose
centre is at x > 0.  These tests build particles at known places, strictly
inside known cells, let the oracle bin them (Eq. signed_histogram), and check
its observables against the particle sums computed here by numpy's
histogram routines and by plain sums over the particles.  The cells are not
square, N_alpha differs from the number of particles, some particles lie
outside the grid, and x = 0 falls on a cell edge in one grid and inside a
cell (in its left or its right half) in the others, so that a missing dk, a
count in place of N_alpha, an edge in place of a centre or a dropped
out-of-grid rule each fail a check.
"""
import numpy as np
import pytest

import oracle


def _particles(rng, nx, nk, xmin, xmax, kmin, kmax, n, n_out):
    """n particles strictly inside random cells (a margin of 5% of the cell
    from every edge) and n_out outside the grid, with random signs."""
    dx, dk = (xmax - xmin) / nx, (kmax - kmin) / nk
    ix = rng.integers(0, nx, n)
    ik = rng.integers(0, nk, n)
    x = xmin + (ix + rng.uniform(0.05, 0.95, n)) * dx
    k = kmin + (ik + rng.uniform(0.05, 0.95, n)) * dk
    xo = np.concatenate([rng.uniform(xmin - 9, xmin - 0.1, n_out // 2),
                         rng.uniform(xmax + 0.1, xmax + 9, n_out - n_out // 2)])
    ko = rng.uniform(kmin + 0.1 * dk, kmax - 0.1 * dk, n_out)
    s = rng.choice([-1.0, 1.0], n + n_out)
    return np.concatenate([x, xo]), np.concatenate([k, ko]), s, ix, ik


@pytest.mark.parametrize("xmin,xmax,nx", [
    (-3.3, 4.9, 24),    # x = 0 in the right half of cell 9: that cell does not count
    (-3.1, 4.9, 24),    # x = 0 in the left half of cell 9: that cell counts
    (-3.0, 5.0, 20),    # x = 0 is the edge between cells 7 and 8
])
def test_observables_equal_the_particle_estimator(xmin, xmax, nx):
    nk, kmin, kmax, n_alpha = 10, -2.0, 3.0, 777
    rng = np.random.default_rng(nx + int(round(-10 * xmin)))
    x, k, s, ix, ik = _particles(rng, nx, nk, xmin, xmax, kmin, kmax, 3000, 200)
    o = oracle.Oracle(nx=nx, nk=nk, xmin=xmin, xmax=xmax, kmin=kmin, kmax=kmax,
                      n_alpha=n_alpha)
    o.set_particles(x, k, s, np.arange(len(x), dtype=np.uint64))
    o.annihilate()
    g = o.grid()
    dens, marg, T = o.observables(g)

    dx, dk = (xmax - xmin) / nx, (kmax - kmin) / nk
    assert dx != dk
    xe = np.linspace(xmin, xmax, nx + 1)
    ke = np.linspace(kmin, kmax, nk + 1)
    # the binning: the signed counts of the particles placed in each cell
    h2, _, _ = np.histogram2d(x, k, bins=[xe, ke], weights=s)
    assert np.array_equal(g, h2.astype(np.int32))
    # density: A = 1{cell} / (dx dk)
    np.testing.assert_allclose(dens, h2 / (n_alpha * dx * dk), rtol=1e-14, atol=0)
    # marginal: A = 1{column} / dx
    h1, _ = np.histogram(x, bins=xe, weights=s)
    np.testing.assert_allclose(marg, h1 / (n_alpha * dx), rtol=1e-14, atol=0)
    # both integrate to the signed mass inside the grid over N_alpha
    inside = (x >= xmin) & (x < xmax)
    mass = s[inside].sum() / n_alpha
    assert abs(dens.sum() * dx * dk - mass) < 1e-12
    assert abs(marg.sum() * dx - mass) < 1e-12
    # transmission: whole cells whose centre is at x > 0, i.e. the particles
    # at or right of that cell's left edge
    j0 = int(np.floor((0.0 - xmin) / dx))          # the cell holding x = 0
    centre0 = xmin + (j0 + 0.5) * dx
    edge = xe[j0] if centre0 > 0 else xe[j0 + 1]
    T_part = s[inside & (x >= edge)].sum() / n_alpha
    assert T == T_part
    if abs(xe[j0]) < 1e-12:   # x = 0 is a cell edge: the estimator of 1{x > 0} itself
        assert T == s[inside & (x > 0)].sum() / n_alpha


def test_observables_of_electron_one_equal_the_particle_estimator():
    """4D: the reduced Wigner function of electron 1 is the estimator with A
    the indicator of an (x1, k1) cell over its measure; the marginal and the
    probability of x1 > 0 likewise, from the counts of a 4D grid whose
    particles are known."""
    nx, nk, n_alpha = 6, 5, 313
    xmin, xmax, kmin, kmax = -2.3, 3.7, -1.0, 1.5   # x = 0 in the left half of cell 2
    rng = np.random.default_rng(11)
    n = 2000
    dx, dk = (xmax - xmin) / nx, (kmax - kmin) / nk
    idx = [rng.integers(0, m, n) for m in (nx, nx, nk, nk)]
    x1 = xmin + (idx[0] + rng.uniform(0.05, 0.95, n)) * dx
    k1 = kmin + (idx[2] + rng.uniform(0.05, 0.95, n)) * dk
    s = rng.choice([-1, 1], n)
    g = np.zeros((nx, nx, nk, nk), np.int64)
    np.add.at(g, tuple(idx), s)
    o = oracle.Oracle4(nx=nx, nk=nk, xmin=xmin, xmax=xmax, kmin=kmin, kmax=kmax,
                       ny=64, nkap=32, n_alpha=n_alpha)
    f1, marg, right = o.observables(g.astype(np.int32))
    h2, _, _ = np.histogram2d(x1, k1, bins=[np.linspace(xmin, xmax, nx + 1),
                                            np.linspace(kmin, kmax, nk + 1)], weights=s)
    np.testing.assert_allclose(f1, h2 / (n_alpha * dx * dk), rtol=1e-14, atol=0)
    h1, _ = np.histogram(x1, bins=np.linspace(xmin, xmax, nx + 1), weights=s)
    np.testing.assert_allclose(marg, h1 / (n_alpha * dx), rtol=1e-14, atol=0)
    assert right == s[x1 >= xmin + 2 * dx].sum() / n_alpha
