"""FP32 candidate clock, checked in law (Sec. 3.2).

Under the constant auxiliary rate gamma0 the first event of a particle in an
interval of length dt falls inside it with probability p = 1 - exp(-gamma0
dt), independently across intervals.  The FP32 path draws the candidate
intervals as geometric gaps: the first of a flight in the flight kernel, each
next one when the event kernel takes the previous one.  With wp every
candidate's first event is logged (its pair weight is nonzero), so the log
shows, per particle, exactly its candidate intervals.  These tests compare
them with independent Bernoulli(p) trials: per-particle counts against the
binomial law, per-interval totals, adjacent pairs, and the same for
regenerated particles and for offspring.
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

WL = workloads.scaled(workloads.COLLISION_2D, precision="fp32", strategy="wp")
P = 1.0 - math.exp(-1.0 * WL["dt"])  # gamma0 = |H|/hbar = 1


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _log(n, steps, resample, seed=3):
    from paper_1709_02121_gb300 import Simulation
    wl = workloads.scaled(WL, n_alpha=n, seed=seed, resample_every=resample)
    sim = Simulation(wl, capacity=40 * n, event_log=6_000_000)
    sim.run(steps)
    ev = sim.event_log()
    assert sim.counters()["log_len"] <= 6_000_000
    sim.close()
    return ev


def _chi2_binom(counts, m, p, zero_truncated=False):
    """Chi-square statistic and dof of counts (one per particle) against
    Binomial(m, p), optionally conditioned on at least one success."""
    ks = np.arange(m + 1)
    pk = np.array([math.comb(m, k) * p ** k * (1 - p) ** (m - k) for k in ks])
    if zero_truncated:
        pk[0] = 0.0
        pk /= pk.sum()
    obs = np.bincount(counts, minlength=m + 1)[: m + 1].astype(float)
    exp = pk * len(counts)
    # pool the tail so that every expected count is at least 20
    lo = 1 if zero_truncated else 0
    o, e = [], []
    acc_o = acc_e = 0.0
    for k in range(lo, m + 1):
        acc_o += obs[k]
        acc_e += exp[k]
        if acc_e >= 20 and exp[k + 1:].sum() >= 20:
            o.append(acc_o)
            e.append(acc_e)
            acc_o = acc_e = 0.0
    o[-1] += acc_o
    e[-1] += acc_e
    o, e = np.array(o), np.array(e)
    return float(np.sum((o - e) ** 2 / e)), len(o) - 1


def _chi2_ok(stat, dof):
    # a 1e-4 tail bound: mean dof, sd sqrt(2 dof), generous for small dof
    return stat < dof + 6.0 * math.sqrt(2.0 * dof) + 10.0


def test_initial_particles_follow_bernoulli_intervals():
    n, steps = 100_000, 12  # two flights (10 + 2 intervals): chains and a restart
    ev = _log(n, steps, 0)
    root = ev[(ev["pid"] < n) & (ev["j"] == 0)]
    # one first event per candidate interval and particle
    key = root["pid"].astype(np.int64) * 64 + root["step"].astype(np.int64)
    assert len(np.unique(key)) == len(root)
    counts = np.bincount(root["pid"].astype(np.int64), minlength=n)
    stat, dof = _chi2_binom(counts, steps, P)
    assert _chi2_ok(stat, dof), (stat, dof)
    per_step = np.bincount(root["step"].astype(np.int64), minlength=steps)
    z = (per_step - n * P) / math.sqrt(n * P * (1 - P))
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    # adjacent intervals are independent: pairs (l, l + 1) at rate p^2,
    # across the flight boundary at l = 9 as well
    s = set(key.tolist())
    pairs = sum(1 for kk in key.tolist() if kk + 1 in s)
    ep = n * (steps - 1) * P * P
    assert abs(pairs - ep) < 4.5 * math.sqrt(ep), (pairs, ep)


def test_regenerated_particles_follow_bernoulli_intervals():
    n, steps, T = 100_000, 15, 5
    ev = _log(n, steps, T)
    base = ev[(ev["pid"] < (1 << 63)) & (ev["j"] == 0) & (ev["step"] >= T)]
    assert len(base) > 10_000
    # regenerated ids carry their epoch: one group per particle and period
    grp = base["pid"].astype(np.uint64)
    _, inv, counts = np.unique(grp, return_inverse=True, return_counts=True)
    assert np.all(np.isin(np.unique(base["step"] // T), [1, 2]))
    stat, dof = _chi2_binom(counts, T, P, zero_truncated=True)
    assert _chi2_ok(stat, dof), (stat, dof)
    # every position in the period equally likely
    pos = np.bincount((base["step"] % T).astype(np.int64), minlength=T).astype(float)
    e = pos.sum() / T
    assert np.sum((pos - e) ** 2 / e) < T - 1 + 6 * math.sqrt(2 * (T - 1)) + 10, pos


def test_offspring_follow_bernoulli_intervals():
    n, steps = 100_000, 12
    ev = _log(n, steps, 0, seed=4)
    born = {}
    for side in ("plus", "minus"):
        alive = ev["kill_" + side] == 0
        for pid, l in zip(ev["pid_" + side][alive].tolist(), ev["step"][alive].tolist()):
            born[pid] = l
    later = ev[(ev["j"] == 0) & (ev["pid"] >= (1 << 63))]
    cnt = {}
    for pid, l in zip(later["pid"].tolist(), later["step"].tolist()):
        if l > born[pid]:
            cnt[pid] = cnt.get(pid, 0) + 1
    # offspring born in interval lb have steps - 1 - lb later intervals: the
    # rest of their first flight (gap from their id) and the next flight
    tot = np.zeros(steps)
    mean = np.zeros(steps)
    var = np.zeros(steps)
    for pid, lb in born.items():
        m = steps - 1 - lb
        tot[lb] += cnt.get(pid, 0)
        mean[lb] += m * P
        var[lb] += m * P * (1 - P)
    ok = var > 100
    assert ok.sum() >= 5
    z = (tot[ok] - mean[ok]) / np.sqrt(var[ok])
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    # the most common birth interval: the full count distribution
    lb = int(np.argmax([sum(1 for v in born.values() if v == b) for b in range(steps)]))
    m = steps - 1 - lb
    if m >= 2:
        c = np.array([cnt.get(pid, 0) for pid, v in born.items() if v == lb])
        stat, dof = _chi2_binom(c, m, P)
        assert _chi2_ok(stat, dof), (stat, dof, lb)
