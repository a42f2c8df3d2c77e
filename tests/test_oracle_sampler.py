"""Pins of the branching law: the candidate clock of constant rate gamma0,
the acceptance (sp1) / weight (sp2) cacc |sin|, and the kick law
V_W^+(x, .)/xi(x) (Alg. 1 item 3 with the majorant reading of Remark 3)."""
import numpy as np
import pytest
from scipy import integrate, stats

import oracle
import workloads
from helpers import make_oracle


def _outcomes(o, x, n):
    emit = np.zeros(n, bool)
    kap = np.zeros(n)
    fac = np.zeros(n)
    gap = np.zeros(n)
    for i in range(n):
        e, k, f, g = o.event_outcome(pid=1000 + i, step=3, j=i % 5, xe=x)
        emit[i], kap[i], fac[i], gap[i] = e, k, f, g
    return emit, kap, fac, gap


@pytest.mark.parametrize("x", [0.3, 1.0, 4.0])
def test_sp1_acceptance_rate_equals_xi_over_gamma0(oracle_mod, x):
    o = make_oracle(workloads.GAUSS_2D_FP64_2E5, n_alpha=10)
    n = 40000
    emit, _, _, _ = _outcomes(o, x, n)
    p = oracle_mod.xi_gauss(1.0, 1.0, 0.0, 1.0, x) / o.gamma0
    se = np.sqrt(p * (1 - p) / n)
    assert abs(emit.mean() - p) < 4.5 * se


@pytest.mark.parametrize("x", [0.4, 1.5])
def test_kick_law_is_positive_part_of_kernel(oracle_mod, x):
    o = make_oracle(workloads.GAUSS_2D_FP64_2E5, n_alpha=10)
    emit, kap, _, _ = _outcomes(o, x, 60000)
    q = kap[emit]
    edges = np.linspace(-2.5, 2.5, 41)
    h, _ = np.histogram(q, bins=edges)
    xi = oracle_mod.xi_gauss(1.0, 1.0, 0.0, 1.0, x)
    pdf = lambda k: max(oracle_mod.vw_gauss(1.0, 1.0, 0.0, 1.0, x, k), 0.0) / xi
    p = np.array([integrate.quad(pdf, a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    exp = p * len(q)
    keep = exp > 10
    chi = np.sum((h[keep] - exp[keep]) ** 2 / exp[keep])
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-3
    # and the kicks carry sign(sin): + child at k + q needs V_W(x, q) > 0
    assert np.all(np.sin(2 * x * q) >= 0)


def test_sp2_weight_factor_mean_and_weighted_kick_law(oracle_mod):
    x = 0.8
    o = make_oracle(workloads.GAUSS_2D_FP64_2E5, n_alpha=10, strategy="sp2")
    emit, kap, fac, _ = _outcomes(o, x, 40000)
    xi = oracle_mod.xi_gauss(1.0, 1.0, 0.0, 1.0, x)
    assert np.all(emit == (fac > 0))
    se = fac.std() / np.sqrt(len(fac))
    assert abs(fac.mean() - xi / o.gamma0) < 4.5 * se
    # weighted kick mean: int q V_W^+(x,q) dq / int V_W^+ dq
    m = integrate.quad(lambda k: k * max(oracle_mod.vw_gauss(1.0, 1.0, 0.0, 1.0, x, k), 0.0),
                       -8, 8, limit=2000)[0] / xi
    est = np.sum(fac * kap) / np.sum(fac)
    assert abs(est - m) < 0.02


def test_gaps_are_exponential_with_rate_gamma0(oracle_mod):
    o = make_oracle(workloads.GAUSS_2D_FP64_2E5, n_alpha=10, gamma0=1.7)
    _, _, _, gap = _outcomes(o, 0.5, 20000)
    assert stats.kstest(gap, "expon", args=(0, 1 / 1.7)).pvalue > 1e-3


def test_accepted_events_per_interval_are_poisson_xi_dt(oracle_mod):
    # far from the barrier xi = 2|H|/(pi hbar); accepted events of a parent
    # in one interval are Poisson(xi dt) by thinning of the gamma0 clock
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, dt=0.4, n_alpha=50000,
                          x0=-30.0, sigma_x=1.0)
    o = make_oracle(wl)
    o.init_gauss(50000, wl["x0"], wl["sigma_x"], wl["k0"])
    o.enable_log()
    o.step(1)
    log = o.event_log()
    par = log[log["pid"] < 50000]
    counts = np.bincount(par["pid"].astype(np.int64), minlength=50000)
    lam = (2 / np.pi) * wl["dt"]
    assert abs(counts.mean() - lam) < 4.5 * np.sqrt(lam / 50000)
    assert abs(counts.var() - lam) < 0.05 * lam
    # event times of parents are uniform over the interval
    assert stats.kstest(par["t"] / wl["dt"], "uniform").pvalue > 1e-3


@pytest.mark.parametrize("H", [-1.0, -0.6, 0.6])
def test_kick_law_follows_the_sign_of_the_potential(oracle_mod, H):
    # Eq. 2: V_W carries the sign of Vhat, i.e. of H.  A well (H < 0) has
    # V_W^+ where H sin(2 (x - xc) q) > 0, so the + child's kick follows
    # max(V_W(x, .), 0)/xi for either sign of H.
    from oracle import refs
    x = 0.7
    o = make_oracle(workloads.GAUSS_2D_FP64_2E5, H=H, n_alpha=10)
    emit, kap, _, _ = _outcomes(o, x, 50000)
    q = kap[emit]
    assert np.all(H * np.sin(2 * x * q) >= 0)
    vw = refs.gauss_vw_closed(H, 1.0, 0.0, 1.0)
    xi = integrate.quad(lambda k: max(vw(x, k), 0.0), -8, 8, limit=2000)[0]
    edges = np.linspace(-2.5, 2.5, 41)
    h, _ = np.histogram(q, bins=edges)
    p = np.array([integrate.quad(lambda k: max(vw(x, k), 0.0) / xi, a, b)[0]
                  for a, b in zip(edges[:-1], edges[1:])])
    exp = p * len(q)
    keep = exp > 10
    chi = np.sum((h[keep] - exp[keep]) ** 2 / exp[keep])
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-3
    # the mean kick of the + child, against an independent Fourier quadrature
    # of the potential itself
    V = refs.gauss_potential(H, 1.0, 0.0)
    qs = np.linspace(-3.0, 3.0, 241)
    vq = np.array([max(refs.vw_quadrature(V, x, k), 0.0) for k in qs])
    m = np.trapezoid(qs * vq, qs) / np.trapezoid(vq, qs)
    assert abs(q.mean() - m) < 5 * q.std() / np.sqrt(len(q)) + 2e-3
