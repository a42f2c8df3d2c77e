"""Pins of the 4D Helium-like oracle (Example 1 with soft-Coulomb terms).

Against what the definitions fix: K0 against a library routine; the tabulated
kernels against the closed form of Eq. 2 (antisymmetry, the total mass
C_m = 2|q_m|/(a hbar), xi_m by quadrature of the continuum kernel); the
branching law (component frequencies, acceptance xi_h/gamma, kick law
V_W^+/xi, kick directions); exact free transport; exact conservation of the
net signed count; the 4D histogram and Alg. 3 by brute force; and the
two-electron Schroedinger equation, whose Wigner transform the method solves.
"""
import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
import workloads
from helpers import make_oracle4
from oracle import refs

WL = workloads.scaled(workloads.HE_4D_FP32_5E7, precision="fp64", n_alpha=2000, nx=16, nk=16)


def kernel(q, a=1.0, hbar=1.0):
    """Continuum V_W of one component from Eq. 2 with Uhat(q) = 2 K0(a|q|)."""
    return lambda y, kap: (4.0 * q / (np.pi * hbar)) * special.k0(2 * a * abs(kap)) * np.sin(2 * y * kap)


def test_k0_against_library():
    for z in np.geomspace(1e-3, 40.0, 60):
        assert abs(oracle.k0(z) / special.k0(z) - 1.0) < 1e-13, z


@pytest.fixture(scope="module")
def o4():
    return make_oracle4(WL)


@pytest.mark.parametrize("t, q", [(0, -2.0), (1, 1.0)])
def test_tables_follow_the_kernel(o4, t, q):
    A, xi, S = o4.table(t, with_S=True)
    K = WL["kmax"] - WL["kmin"]
    dkap = 2 * K / WL["nkap"]
    kap = -K + (np.arange(WL["nkap"]) + 0.5) * dkap
    assert np.allclose(A, (4 * q / np.pi) * special.k0(2 * np.abs(kap)), rtol=1e-13, atol=0)
    # symmetric kappa mesh: A even, so V_W(y, -kappa) = -V_W(y, kappa) and
    # xi = (1/2) dkappa sum |V_W|
    assert np.allclose(A, A[::-1], rtol=1e-12, atol=0)
    Y = (1 if t == 0 else 2) * (WL["xmax"] - WL["xmin"])
    y = -Y + np.arange(WL["ny"]) * (2 * Y / (WL["ny"] - 1))
    for i in (0, 7, 1500, 2047, 2048, 3333, 4095):
        vw = A * np.sin(2 * y[i] * kap)
        assert abs(xi[i] - 0.5 * dkap * np.abs(vw).sum()) <= 1e-12 * max(xi[i], 1e-300)
        v = np.diff(np.concatenate([[0.0], S[i]]))
        # (differences of prefix sums: absolute error ~ rounding of the sum)
        assert np.all(v >= 0)
        assert np.allclose(v, np.maximum(vw, 0), rtol=1e-9, atol=1e-13 * S[i, -1])
    # total mass of |V_W| over kappa: C = 2|q|/(a hbar), less the midpoint
    # rule's deficit at the logarithmic singularity of K0 (two cells of
    # -ln|kappa|: dkappa (1 - ln 2) 4a/pi relative, 0.5% here)
    ratio = np.abs(A).sum() * dkap / (2 * abs(q))
    assert 0.0 < 1.0 - ratio < 1.3 * dkap * (1 - np.log(2)) * 4 / np.pi
    # rate: the smallest multiple of 2^-10 at or above max xi
    g = o4.gamma(t)
    assert g >= xi.max() and g - xi.max() < 2 ** -10 and g * 1024 == round(g * 1024)


@pytest.mark.parametrize("t, q, y", [(0, -2.0, 0.37), (0, -2.0, 3.1), (1, 1.0, -5.2), (1, 1.0, 17.0)])
def test_xi_against_continuum_quadrature(o4, t, q, y):
    A, xi = o4.table(t)
    Y = (1 if t == 0 else 2) * (WL["xmax"] - WL["xmin"])
    dy = 2 * Y / (WL["ny"] - 1)
    s = (y + Y) / dy
    i = int(np.floor(s))
    th = s - i
    xi_h = (1 - th) * xi[i] + th * xi[i + 1]
    vw = kernel(q)
    ref = integrate.quad(lambda k: max(vw(y, k), 0.0), 0, 12.8, limit=4000, points=[0.0])[0] \
        + integrate.quad(lambda k: max(vw(y, k), 0.0), -12.8, 0, limit=4000)[0]
    assert abs(xi_h / ref - 1.0) < 3e-3, (xi_h, ref)


def _events(o, x1e, x2e, n, step=3):
    rows = [o.event_outcome(pid=5000 + i, step=step, j=i % 3, x1e=x1e, x2e=x2e) for i in range(n)]
    emit = np.array([r[0] for r in rows])
    comp = np.array([r[1] for r in rows])
    kap = np.array([r[2] for r in rows])
    prob = np.array([r[3] for r in rows])
    gap = np.array([r[4] for r in rows])
    return emit, comp, kap, prob, gap


def test_component_choice_acceptance_and_gaps(o4):
    n = 60000
    emit, comp, kap, prob, gap = _events(o4, 1.3, -0.6, n)
    G = o4.Gamma
    g = np.array([o4.gamma(0), o4.gamma(0), o4.gamma(1)])
    h = np.bincount(comp, minlength=3)
    chi = np.sum((h - n * g / G) ** 2 / (n * g / G))
    assert stats.chi2.sf(chi, 2) > 1e-3
    for m in range(3):
        sel = comp == m
        p = prob[sel][0]
        assert np.all(prob[sel] == p)
        se = np.sqrt(p * (1 - p) / sel.sum())
        assert abs(emit[sel].mean() - p) < 4.5 * se
    # the gaps are exponential with rate Gamma
    assert stats.kstest(gap, "expon", args=(0, 1 / G)).pvalue > 1e-3


@pytest.mark.parametrize("m, x1e, x2e", [(0, 1.3, -0.6), (1, 1.3, -0.6), (2, 2.2, -0.4)])
def test_kick_law_is_the_positive_part_of_the_component(o4, m, x1e, x2e):
    n = 90000
    emit, comp, kap, prob, gap = _events(o4, x1e, x2e, n)
    q = kap[emit & (comp == m)]
    y = [x1e, x2e, x1e - x2e][m]
    vw = kernel(-2.0 if m < 2 else 1.0)
    edges = np.linspace(-3.0, 3.0, 31)
    xi = sum(integrate.quad(lambda k: max(vw(y, k), 0.0), a, b, limit=400)[0]
             for a, b in zip(edges[:-1], edges[1:]))
    p = np.array([integrate.quad(lambda k: max(vw(y, k), 0.0), a, b, limit=400)[0]
                  for a, b in zip(edges[:-1], edges[1:])]) / xi
    hist, _ = np.histogram(q, bins=edges)
    keep = (p * hist.sum()) > 10
    e = p[keep] * hist[keep].sum() / p[keep].sum()
    chi = np.sum((hist[keep] - e) ** 2 / e)
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-3
    # every kick lies where the component's V_W is positive
    assert np.all(np.sign(vw(y, q)) >= 0) or np.mean(vw(y, q) < 0) < 2e-3


def test_kick_directions_and_pair_signs():
    o = make_oracle4(WL, n_alpha=3000)
    o.enable_log()
    o.init_gauss(3000, WL["x0"], WL["sigma_x"], WL["k0"])
    x1, x2, k1, k2, w, pid = o.particles()
    parent = dict(zip(pid.tolist(), zip(k1, k2)))
    o.step(1)
    log = o.event_log()
    assert len(log) > 100 and set(np.unique(log["comp"])) == {0, 1, 2}
    X1, X2, K1, K2, W, P = o.particles()
    child = dict(zip(P.tolist(), zip(K1, K2, W)))
    d = {0: (1, 0), 1: (0, 1), 2: (1, -1)}
    checked = 0
    for e in log:
        if e["pid"] not in parent:
            continue
        pk1, pk2 = parent[e["pid"]]
        e1, e2 = d[int(e["comp"])]
        for cp, sgn in ((e["pid_plus"], 1), (e["pid_minus"], -1)):
            if cp in child:
                ck1, ck2, cw = child[cp]
                assert ck1 == pk1 + sgn * e1 * e["kappa"] and ck2 == pk2 + sgn * e2 * e["kappa"]
                assert cw == sgn
                checked += 1
    assert checked > 100


def test_free_transport_is_exact():
    o = make_oracle4(WL, Z=0.0, lam=0.0, n_alpha=500)
    o.init_gauss(500, WL["x0"], WL["sigma_x"], WL["k0"])
    x1, x2, k1, k2, w, pid = o.particles()
    dtv = WL["dt"] * WL["hbar"] / WL["mass"]
    for _ in range(7):
        x1, x2 = x1 + k1 * dtv, x2 + k2 * dtv
    o.step(7)
    y1, y2, q1, q2, ww, pp = o.particles()
    assert np.array_equal(pp, pid) and np.array_equal(y1, x1) and np.array_equal(y2, x2)
    assert np.array_equal(q1, k1) and np.array_equal(q2, k2) and np.all(ww == 1)


def test_net_sign_is_conserved_up_to_kills():
    o = make_oracle4(WL, n_alpha=1500)
    o.init_gauss(1500, WL["x0"], WL["sigma_x"], WL["k0"])
    o.step(12)
    w = o.particles()[4]
    led = o.ledger()
    assert led["events"] > 100
    assert int(np.sum(w)) == 1500 - (led["kill_plus"] - led["kill_minus"])


def test_histogram_and_regeneration_by_brute_force():
    o = make_oracle4(WL, n_alpha=1500)
    o.init_gauss(1500, WL["x0"], WL["sigma_x"], WL["k0"])
    o.step(6)
    x1, x2, k1, k2, w, _ = o.particles()
    dx = (WL["xmax"] - WL["xmin"]) / WL["nx"]
    dk = (WL["kmax"] - WL["kmin"]) / WL["nk"]
    i = [np.floor((x1 - WL["xmin"]) * (1 / dx)), np.floor((x2 - WL["xmin"]) * (1 / dx)),
         np.floor((k1 - WL["kmin"]) * (1 / dk)), np.floor((k2 - WL["kmin"]) * (1 / dk))]
    n = [WL["nx"], WL["nx"], WL["nk"], WL["nk"]]
    ok = np.all([(a >= 0) & (a < m) for a, m in zip(i, n)], axis=0)
    ref = np.zeros(n, np.int64)
    np.add.at(ref, tuple(a[ok].astype(int) for a in i), np.sign(w[ok]).astype(int))
    o.annihilate()
    g = o.grid()
    assert np.array_equal(g, ref)
    # Alg. 3: |c| particles of sign(c) per cell, each inside its cell
    y1, y2, q1, q2, ww, pid = o.particles()
    assert len(ww) == np.abs(g).sum()
    j = [np.floor((y1 - WL["xmin"]) * (1 / dx)), np.floor((y2 - WL["xmin"]) * (1 / dx)),
         np.floor((q1 - WL["kmin"]) * (1 / dk)), np.floor((q2 - WL["kmin"]) * (1 / dk))]
    back = np.zeros(n, np.int64)
    np.add.at(back, tuple(a.astype(int) for a in j), ww.astype(int))
    assert np.array_equal(back, g)
    assert np.array_equal(pid & np.uint64(0xFFFFFFFFFF), np.arange(len(pid), dtype=np.uint64))
    # observables of electron 1 by a plain reduction
    f1, marg, right = o.observables(g)
    red = g.sum(axis=(1, 3))
    assert np.allclose(f1, red / (1500 * dx * dk), rtol=1e-15, atol=0)
    centres = WL["xmin"] + (np.arange(WL["nx"]) + 0.5) * dx
    assert right == red[centres > 0].sum() / 1500


def test_matches_the_two_electron_schroedinger_equation():
    # pure branching (no resampling) to t = 0.4: the Monte Carlo estimate of
    # electron 1's position density against a split-step solution of the
    # two-electron TDSE with the same potential and initial packets
    edges = np.linspace(-5.0, 3.0, 9)
    V = refs.soft_coulomb_2e(2.0, 1.0, 1.0)
    x, r1, r2 = refs.tdse2_marginals(V, WL["x0"], WL["sigma_x"], WL["k0"], 0.4)
    ref = refs.bin_density(x, r1, edges)
    cells = []
    n = 40000
    for seed in range(6):
        o = make_oracle4(WL, n_alpha=n, seed=seed)
        o.init_gauss(n, WL["x0"], WL["sigma_x"], WL["k0"])
        o.step(20)
        x1, x2, k1, k2, w, _ = o.particles()
        h, _ = np.histogram(x1, bins=edges, weights=w)
        cells.append(h / n)
    cells = np.array(cells)
    m, se = cells.mean(0), cells.std(0, ddof=1) / np.sqrt(len(cells))
    z = (m - ref) / np.sqrt(se ** 2 + 1e-8)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.mean(z ** 2) < 3.0, np.round(z, 2)
