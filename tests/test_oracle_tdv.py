"""Pins of the oracle with a time-dependent potential (Remark 1).

V(x, t) = sum_m (a_m + b_m cos(om_m t + ph_m)) exp(-(x - xc_m)^2/(2 w_m^2)),
each component with its own majorant rate (|a_m| + |b_m|)/hbar, a death
picking a component in proportion to its rate and accepting with the
component's majorant ratio at the event's absolute time.  Pinned by: a
single static component reproducing the static run bit for bit; the net
sign conserved up to kills; and the Schroedinger equation with the same
potential, static double barrier and time-varying barrier.
"""
import numpy as np
import pytest

import workloads
from helpers import make_oracle
from oracle import refs

WL = workloads.COLLISION_2D
EDGES = np.linspace(-8.0, 8.0, 17)


def run(wl, steps, n=None, **over):
    n = n or wl["n_alpha"]
    o = make_oracle(wl, n_alpha=n, **over)
    o.init_gauss(n, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(steps)
    return o


def test_one_static_component_is_the_static_run():
    a = run(WL, 8, n=3000)
    b = run(WL, 8, n=3000, comps=[dict(a=WL["H"], b=0.0, om=0.0, ph=0.0, w=WL["w"],
                                       xc=WL["xc"])])
    for u, v in zip(a.particles(), b.particles()):
        assert np.array_equal(u, v)
    assert a.ledger() == b.ledger()


def test_net_sign_is_conserved_up_to_kills():
    comps = [dict(a=0.4, b=0.4, om=3.0, ph=np.pi, w=1.0, xc=-1.0),
             dict(a=0.8, b=0.0, om=0.0, ph=0.0, w=0.7, xc=2.0)]
    o = run(WL, 10, n=4000, comps=comps)
    w = o.particles()[2]
    led = o.ledger()
    assert led["events"] > 500
    assert int(np.sum(w)) == 4000 - (led["kill_plus"] - led["kill_minus"])


def _mc(comps, steps, nrep=8, n=20000):
    cells = []
    for seed in range(nrep):
        o = run(WL, steps, n=n, seed=seed, comps=comps)
        x, k, w, _ = o.particles()
        h, _ = np.histogram(x, bins=EDGES, weights=w)
        cells.append(h / n)
    cells = np.array(cells)
    return cells.mean(0), cells.std(0, ddof=1) / np.sqrt(nrep)


@pytest.mark.parametrize("comps", [
    # a static double barrier
    [dict(a=0.8, b=0.0, om=0.0, ph=0.0, w=0.6, xc=-0.5), dict(a=0.5, b=0.0, om=0.0, ph=0.0,
                                                              w=0.8, xc=1.5)],
    # a barrier switched on and off: 0.6 (1 + cos(3 t + 2))
    [dict(a=0.6, b=0.6, om=3.0, ph=2.0, w=1.0, xc=0.0)],
])
def test_matches_the_schroedinger_equation(comps):
    Vt = refs.gauss_components(comps)
    x, rho = refs.tdse_density_t(Vt, WL["x0"], WL["sigma_x"], WL["k0"], 2.0, L=80.0, n=4096,
                                 dt=2e-3)
    ref = refs.bin_density(x, rho, EDGES)
    m, se = _mc(comps, 20)
    z = (m - ref) / np.sqrt(se ** 2 + 1e-8)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.mean(z ** 2) < 2.5, np.round(z, 2)


def test_time_dependence_is_visible():
    # the same barrier frozen at its time-averaged height differs from the
    # switched one by much more than the Monte Carlo error (the pin above
    # would not notice a clock that ignored the absolute time otherwise)
    sw = [dict(a=0.6, b=0.6, om=3.0, ph=np.pi, w=1.0, xc=0.0)]
    fr = [dict(a=0.6, b=0.0, om=0.0, ph=0.0, w=1.0, xc=0.0)]
    ms, ses = _mc(sw, 20, nrep=4)
    mf, sef = _mc(fr, 20, nrep=4)
    z = (ms - mf) / np.sqrt(ses ** 2 + sef ** 2 + 1e-8)
    assert np.max(np.abs(z)) > 6.0
