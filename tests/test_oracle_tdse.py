"""The whole method against quantum mechanics: for a pure state the Wigner
equation (Eq. 1) is the Schroedinger equation, so the oracle's estimates of
the position density and of the transmission (Eq. estimator) must agree with
a split-step solution of the TDSE within their Monte Carlo errors.  The
deterministic grid solver of the truncated Wigner equation is checked against
the same TDSE and then serves as a second reference."""
import numpy as np
import pytest

import workloads
from helpers import make_oracle
from oracle import refs

WL = workloads.COLLISION_2D
EDGES = np.linspace(-8.0, 8.0, 17)
T_END = 2.0


@pytest.fixture(scope="module")
def tdse():
    V = refs.gauss_potential(WL["H"], WL["w"], WL["xc"])
    x, rho = refs.tdse_density(V, WL["x0"], WL["sigma_x"], WL["k0"], T_END,
                               L=80.0, n=4096, dt=2e-3)
    cells = refs.bin_density(x, rho, EDGES)
    T = refs.bin_density(x, rho, np.array([0.0, 40.0 - 1e-9]))[0]
    return x, rho, cells, T


@pytest.fixture(scope="module")
def grid_solution():
    V = refs.gauss_potential(WL["H"], WL["w"], WL["xc"])
    g = refs.GridWigner(V, xa=-12, xb=12, nx=160, ka=-3.5, kb=4.5, nk=128,
                        vw=refs.gauss_vw_closed(WL["H"], WL["w"], WL["xc"], 1.0))
    X, K = np.meshgrid(g.x, g.k, indexing="ij")
    f0 = refs.wigner_gauss_f0(X, K, WL["x0"], WL["sigma_x"], WL["k0"])
    f = g.run(f0, T_END, 0.05)
    marg = f.sum(1) * g.dk
    T = marg[g.x > 0].sum() * g.dx + 0.5 * marg[g.x == 0].sum() * g.dx
    return g.x, marg, T


def _mc(strategy, nrep=8, resample=0, steps=20, **over):
    cells, Ts = [], []
    for seed in range(nrep):
        o = make_oracle(WL, seed=seed, strategy=strategy, **over)
        o.init_gauss(WL["n_alpha"], WL["x0"], WL["sigma_x"], WL["k0"])
        for s in range(steps):
            o.step(1)
            if resample and (s + 1) % resample == 0 and s + 1 < steps:
                o.annihilate()
        x, k, w, _ = o.particles()
        h, _ = np.histogram(x, bins=EDGES, weights=w)
        cells.append(h / WL["n_alpha"])
        Ts.append(np.sum(w[x > 0]) / WL["n_alpha"])
    cells, Ts = np.array(cells), np.array(Ts)
    return (cells.mean(0), cells.std(0, ddof=1) / np.sqrt(nrep),
            Ts.mean(), Ts.std(ddof=1) / np.sqrt(nrep))


def _check(m, se, ref, T, Tse, Tref, bias=0.0):
    z = (m - ref) / np.sqrt(se ** 2 + 1e-8)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.mean(z ** 2) < 2.5, np.round(z, 2)
    assert abs(T - Tref) < 4.0 * Tse + bias, (T, Tse, Tref)


def test_grid_solver_matches_tdse(tdse, grid_solution):
    x, rho, _, Tref = tdse
    gx, marg, Tg = grid_solution
    assert np.max(np.abs(marg - np.interp(gx, x, rho))) < 2e-4
    assert abs(Tg - Tref) < 1e-3


def test_sp1_pure_branching_matches_tdse(tdse):
    _, _, ref, Tref = tdse
    m, se, T, Tse = _mc("sp1")
    _check(m, se, ref, T, Tse, Tref)


def test_sp1_matches_grid_solver(grid_solution):
    gx, marg, Tg = grid_solution
    m, se, T, Tse = _mc("sp1", nrep=6)
    ref = refs.bin_density(gx, marg, EDGES)
    z = (m - ref) / np.sqrt(se ** 2 + 1e-8)
    assert np.max(np.abs(z)) < 4.5
    assert abs(T - Tg) < 4.0 * Tse + 1e-3


def test_sp1_with_annihilation_matches_tdse(tdse):
    _, _, ref, Tref = tdse
    m, se, T, Tse = _mc("sp1", resample=5, nx=320, nk=256)
    _check(m, se, ref, T, Tse, Tref, bias=0.004)


def test_wp_propagation_matches_tdse(tdse):
    # sp2 without a filter is the weighted-particle walk wp
    _, _, ref, Tref = tdse
    m, se, T, Tse = _mc("sp2", nrep=6, steps=20, n_alpha=6000)
    _check(m, se, ref, T, Tse, Tref)


def test_sp2_with_bootstrap_matches_tdse(tdse):
    _, _, ref, Tref = tdse
    m, se, T, Tse = _mc("sp2", resample=5, nx=320, nk=256)
    _check(m, se, ref, T, Tse, Tref, bias=0.004)
