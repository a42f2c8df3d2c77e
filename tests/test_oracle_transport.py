"""Free transport pins: with V = 0 the Wigner equation is pure streaming,
f(x,k,t) = f0(x - hbar k t/m, k) (Eq. 1 with Theta_V = 0)."""
import numpy as np
from scipy import integrate, special

import workloads
from helpers import make_oracle


def _free_oracle(n=4000, steps=7, **over):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, H=0.0, gamma0=1.0,
                          n_alpha=n, **over)
    o = make_oracle(wl)
    o.init_gauss(n, wl["x0"], wl["sigma_x"], wl["k0"])
    return o, wl


def test_no_events_without_potential(oracle_mod):
    o, _ = _free_oracle()
    o.step(7)
    led = o.ledger()
    assert led["events"] == 0 and o.n == 4000
    assert led["particle_steps"] == 7 * 4000


def test_exact_free_streaming(oracle_mod):
    o, wl = _free_oracle(dt=0.1)
    x0, k0, _, pid0 = o.particles()
    o.step(7)
    x, k, w, pid = o.particles()
    assert np.array_equal(pid, pid0) and np.array_equal(k, k0)
    assert np.all(w == 1.0)
    # the specified operation sequence: x <- x + k*dtv, one rounding each
    xs = x0.copy()
    dtv = wl["dt"] * wl["hbar"] / wl["mass"]
    for _ in range(7):
        xs = xs + k0 * dtv
    assert np.array_equal(x, xs)
    # and the exact trajectory x0 + k t to FP64 accuracy
    exact = x0 + k0 * (7 * wl["dt"])
    assert np.max(np.abs(x - exact) / np.maximum(1.0, np.abs(exact))) < 1e-12


def test_mass_ratio_scales_velocity(oracle_mod):
    o, wl = _free_oracle(mass=2.0, hbar=0.5)
    x0, k0, _, _ = o.particles()
    o.step(3)
    x, _, _, _ = o.particles()
    exact = x0 + k0 * (0.5 / 2.0) * (3 * wl["dt"])
    assert np.max(np.abs(x - exact)) < 1e-12 * 20


def test_transported_histogram_matches_cell_integrals(oracle_mod):
    # f(x,k,t) = f0(x - k t, k): its cell integrals vs the oracle's histogram
    n, steps = 200000, 30
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, H=0.0, gamma0=1.0,
                          n_alpha=n, nx=60, nk=16, xmin=-30.0, xmax=30.0,
                          kmin=0.7, kmax=2.3)
    o = make_oracle(wl)
    o.init_gauss(n, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(steps)
    counts, _ = o.histogram()
    t = steps * wl["dt"]
    sx, sk = wl["sigma_x"], 1.0 / (2 * wl["sigma_x"])
    xe = np.linspace(wl["xmin"], wl["xmax"], wl["nx"] + 1)
    ke = np.linspace(wl["kmin"], wl["kmax"], wl["nk"] + 1)
    p = np.zeros((wl["nx"], wl["nk"]))
    for j in range(wl["nk"]):
        for i in range(wl["nx"]):
            g = lambda k: (np.exp(-((k - wl["k0"]) ** 2) / (2 * sk * sk)) / (np.sqrt(2 * np.pi) * sk)
                           * 0.5 * (special.erf((xe[i + 1] - k * t - wl["x0"]) / (np.sqrt(2) * sx))
                                    - special.erf((xe[i] - k * t - wl["x0"]) / (np.sqrt(2) * sx))))
            p[i, j] = integrate.quad(g, ke[j], ke[j + 1])[0]
    expect = n * p
    se = np.sqrt(n * p * (1 - p)) + 1e-12
    z = (counts - expect) / se
    big = expect > 25
    assert big.sum() > 100
    assert np.max(np.abs(z[big])) < 5.0
    assert abs(np.mean(z[big] ** 2) - 1.0) < 0.25
