"""Pins of the oracle's wp resampling (weighted particles, Sec. 4.3).

wp propagates weighted particles (pairs always made, weights +/- w cacc
|sin|, as sp2 between its filters) and resamples by the weighted histogram
of Eq. piecewise_constant_function followed by Alg. 3 with its rounding
step.  Pinned by: the counts against the particles' fixed-point weight sums
(brute force, exact), the unbiased rounding in law, and the TDSE.
"""
import numpy as np

import workloads
from helpers import make_oracle
from oracle import refs

WL = workloads.scaled(workloads.COLLISION_2D, strategy="wp")


def run(steps, n=4000, seed=0, resample=0):
    o = make_oracle(WL, n_alpha=n, seed=seed)
    o.init_gauss(n, WL["x0"], WL["sigma_x"], WL["k0"])
    for s in range(steps):
        o.step(1)
        if resample and (s + 1) % resample == 0 and s + 1 < steps:
            o.annihilate()
    return o


def test_counts_round_each_cells_weight_sum():
    o = run(6)
    x, k, w, _ = o.particles()
    assert np.any((w != 0) & (np.abs(w) < 1))     # weighted offspring exist
    dx = (WL["xmax"] - WL["xmin"]) / WL["nx"]
    dk = (WL["kmax"] - WL["kmin"]) / WL["nk"]
    ix = np.floor((x - WL["xmin"]) * (1 / dx)).astype(int)
    ik = np.floor((k - WL["kmin"]) * (1 / dk)).astype(int)
    ok = (ix >= 0) & (ix < WL["nx"]) & (ik >= 0) & (ik < WL["nk"])
    ws = np.zeros((WL["nx"], WL["nk"]), np.int64)
    np.add.at(ws, (ix[ok], ik[ok]), np.rint(w[ok] * 2.0 ** 31).astype(np.int64))
    o.annihilate()
    g = o.grid()
    m = ws * 2.0 ** -31
    assert np.all(np.abs(g) >= np.floor(np.abs(m))) and np.all(np.abs(g) <= np.ceil(np.abs(m)))
    assert np.all((g == 0) | (np.sign(g) == np.sign(m)))
    # the rounding is unbiased: the round-ups match the fractional parts
    frac = np.abs(m) - np.floor(np.abs(m))
    ups = np.abs(g) - np.floor(np.abs(m))
    sel = frac > 0
    n = sel.sum()
    assert n > 300
    assert abs(ups[sel].sum() - frac[sel].sum()) < 4.5 * np.sqrt((frac[sel] * (1 - frac[sel])).sum())


def test_wp_with_resampling_matches_the_schroedinger_equation():
    edges = np.linspace(-8.0, 8.0, 17)
    V = refs.gauss_potential(WL["H"], WL["w"], WL["xc"])
    x, rho = refs.tdse_density(V, WL["x0"], WL["sigma_x"], WL["k0"], 2.0, L=80.0, n=4096, dt=2e-3)
    ref = refs.bin_density(x, rho, edges)
    cells = []
    n = 20000
    for seed in range(8):
        o = run(20, n=n, seed=seed, resample=5)
        xs, ks, w, _ = o.particles()
        cells.append(np.histogram(xs, bins=edges, weights=w)[0] / n)
    cells = np.array(cells)
    mean, se = cells.mean(0), cells.std(0, ddof=1) / np.sqrt(len(cells))
    z = (mean - ref) / np.sqrt(se ** 2 + 1e-8)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.mean(z ** 2) < 3.0, np.round(z, 2)
