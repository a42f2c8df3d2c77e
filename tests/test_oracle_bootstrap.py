"""Pins of the signed residual bootstrap (Alg. 2 on S+ and S-, Eq. lambda,
Eq. double_bootstrap) and of the rounding step of Alg. 3, on inputs small
enough to enumerate the exact law of the filtered counts."""
from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np
import pytest
from scipy import stats

import workloads
from helpers import make_oracle

# three cells along x, one along k
GRID = dict(nx=3, nk=1, xmin=0.0, xmax=3.0, kmin=0.0, kmax=1.0)
WPOS = [0.9, 0.35, 0.6, 0.15, 0.5]
CPOS = [0, 0, 1, 2, 2]
WNEG = [-0.7, -0.2, -0.45]
CNEG = [1, 2, 0]


def _particles():
    w = np.array(WPOS + WNEG)
    cells = np.array(CPOS + CNEG)
    x = cells + 0.5
    k = np.full(len(w), 0.5)
    pid = np.arange(len(w), dtype=np.uint64)
    return x, k, w, pid


def _exact_law(weights, cells, ncell=3):
    """Law of the filtered counts by cell from Alg. 2 in exact arithmetic:
    q_i = |w_i| N / sum|w|, keep floor(q_i) copies, then N_r draws with
    probabilities proportional to the residuals q_i - floor(q_i)."""
    N = len(weights)
    aw = [Fraction(abs(w)).limit_denominator(10 ** 12) for w in weights]
    W = sum(aw)
    q = [a * N / W for a in aw]
    keep = [0] * ncell
    res = [Fraction(0)] * ncell
    for qi, c in zip(q, cells):
        fl = qi.numerator // qi.denominator
        keep[c] += fl
        res[c] += qi - fl
    nr = N - sum(keep)
    R = sum(res)
    p = [r / R for r in res]
    law = {}
    for comp in product(range(nr + 1), repeat=ncell):
        if sum(comp) != nr:
            continue
        pr = Fraction(factorial(nr))
        for ci, pi in zip(comp, p):
            pr = pr * pi ** ci / factorial(ci)
        law[tuple(k + c for k, c in zip(keep, comp))] = float(pr)
    mean = [float(sum(qi for qi, c in zip(q, cells) if c == nu)) for nu in range(ncell)]
    return law, mean, nr


@pytest.fixture(scope="module")
def trials():
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, strategy="sp2",
                          n_alpha=4, **GRID)
    o = make_oracle(wl)
    x, k, w, pid = _particles()
    plus, minus, grids = [], [], []
    for _ in range(20000):
        o.set_particles(x, k, w, pid)
        o.annihilate()
        p, m = o.boot_counts()
        plus.append(p[:, 0].copy())
        minus.append(m[:, 0].copy())
        grids.append(o.grid()[:, 0].copy())
    return np.array(plus), np.array(minus), np.array(grids), o.boot_stats()


@pytest.mark.parametrize("side", ["plus", "minus"])
def test_filtered_counts_follow_exact_law(trials, side):
    plus, minus, _, _ = trials
    data = plus if side == "plus" else minus
    wts, cls = (WPOS, CPOS) if side == "plus" else (WNEG, CNEG)
    law, mean, nr = _exact_law(wts, cls)
    assert nr > 0
    assert np.all(data.sum(1) == len(wts))        # sum_nu n~_nu = N^s
    keys = list(law)
    obs = np.array([np.sum(np.all(data == np.array(k), axis=1)) for k in keys])
    assert obs.sum() == len(data)                  # no impossible outcome
    exp = np.array([law[k] for k in keys]) * len(data)
    big = exp > 5
    chi = np.sum((obs[big] - exp[big]) ** 2 / exp[big])
    assert stats.chi2.sf(chi, big.sum() - 1) > 1e-3
    se = data.std(0) / np.sqrt(len(data))
    assert np.all(np.abs(data.mean(0) - mean) < 4.5 * se + 1e-9)


def test_bootstrap_variance_bounds(trials):
    # Lemma 1 on each side and Theorem 2 for the signed measure, with
    # phi = indicator of one cell (||phi|| = 1)
    plus, minus, _, st = trials
    Np, Nm = len(WPOS), len(WNEG)
    Wp, Wm = sum(WPOS), -sum(WNEG)
    na = 1.0
    lam_p, lam_m = Wp / na, -Wm / na
    for nu in range(3):
        exact_p = sum(w for w, c in zip(WPOS, CPOS) if c == nu) / Wp
        err_p = plus[:, nu] / Np - exact_p
        nr_p = st["nr"][0]
        assert np.mean(err_p ** 2) <= 2 * (nr_p / Np + 1) / Np
        exact = (sum(w for w, c in zip(WPOS + WNEG, CPOS + CNEG) if c == nu)) / na
        est = lam_p * plus[:, nu] / Np + lam_m * minus[:, nu] / Nm
        assert np.mean((exact - est) ** 2) <= 8 * (lam_p ** 2 / Np + lam_m ** 2 / Nm)


def test_rounding_step_of_alg3(trials):
    plus, minus, grids, st = trials
    Np, Nm = len(WPOS), len(WNEG)
    wfix = st["wfix"].astype(np.float64) / 2.0 ** 31
    m = plus * (wfix[0] / Np) - minus * (wfix[1] / Nm)
    n = np.abs(grids)
    fl = np.floor(np.abs(m))
    assert np.all((n == fl) | (n == fl + 1))
    assert np.all((grids == 0) | (np.sign(grids) == np.sign(m)))
    frac = np.abs(m) - fl
    d = (n - fl) - frac                      # E[n - |m|] = 0
    assert abs(d.mean()) < 4.5 * d.std() / np.sqrt(d.size) + 1e-12


def test_sp1_rounding_is_skipped(oracle_mod):
    # sp1: m is an integer count, Alg. 3's rounding never changes it
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=4, **GRID)
    o = make_oracle(wl)
    x, k, w, pid = _particles()
    o.set_particles(x, k, np.sign(w), pid)
    o.annihilate()
    assert o.grid()[:, 0].tolist() == [2 - 1, 1 - 1, 2 - 1]
