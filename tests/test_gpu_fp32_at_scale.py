"""FP32 accuracy at the scale the benchmark times: the 2D Gaussian barrier on
the 1200 x 512 grid over x in [-60, 60), k in [-6.4, 6.4), dt = 0.05,
resampling every 10 intervals, to t = 20 (400 intervals).

The FP64 path is bit-identical to the oracle (the parity tests), so it is the
reference here.  Both paths estimate the same expectation on the same grid
with the same resampling, so the resampling bias of Theorem 3 is common to
both and cancels; what is left is the Monte Carlo error, which 16 independent
runs of 1e7 particles on each side measure.  Compared:

- the phase-space density (Eq. signed_histogram over N_alpha and the cell
  measure) re-binned to 60 x 32 blocks of 20 x 16 cells, at t = 10 and
  t = 20, cell by cell in units of the combined standard error: the number
  of cells beyond 3 standard errors must agree with the rate that the
  t-distribution of the 16 + 16 runs gives, no cell may pass the Bonferroni
  bound of the whole family, and the mean squared deviation must stay near
  its null value;
- the transmission (Eq. estimator with A = 1{x > 0}) within 2e-3 absolute,
  with a standard error small enough for that to mean something.

One run at the benchmark's full size (1e8 particles, the same capacity,
CUDA-graph replay) is compared with the same reference, its variance taken
as a tenth of a 1e7 run's (Monte Carlo variance goes as 1/N_alpha).
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

WL = workloads.GAUSS_2D_FP32_1E8
N = 10_000_000
SEEDS = 16
BLOCK = (20, 16)          # cells per block: 1200 x 512 -> 60 x 32
TIMES = (200, 400)        # intervals: t = 10 and t = 20


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def _blocks(g):
    nx, nk = g.shape
    bx, bk = BLOCK
    return g.reshape(nx // bx, bx, nk // bk, bk).sum(axis=(1, 3), dtype=np.int64)


def _run(torch, precision, n, seed, graphs=False, capacity_factor=4.0):
    """Densities of the re-binned blocks and transmissions at TIMES."""
    from paper_1709_02121_gb300 import Simulation
    wl = workloads.scaled(WL, precision=precision, n_alpha=n, seed=seed)
    sim = Simulation(wl, capacity=int(capacity_factor * n) + (1 << 20),
                     stream=torch.cuda.Stream())
    if graphs:
        sim.graph(True)
    dx = (wl["xmax"] - wl["xmin"]) / wl["nx"] * BLOCK[0]
    dk = (wl["kmax"] - wl["kmin"]) / wl["nk"] * BLOCK[1]
    dens, Ts, live = [], [], []
    done = 0
    for t in TIMES:
        sim.run(t - done)
        done = t
        _, _, T, n_live = sim.density()
        dens.append(_blocks(sim.grid_counts()) / (n * dx * dk))
        Ts.append(T)
        live.append(n_live)
    assert sim.counters()["error"] == 0
    sim.close()
    return np.array(dens), np.array(Ts), live


@pytest.fixture(scope="module")
def runs(torch):
    out = {}
    for prec, base in (("fp32", 0), ("fp64", 1000)):
        d, T = [], []
        for s in range(SEEDS):
            di, Ti, _ = _run(torch, prec, N, base + s)
            d.append(di)
            T.append(Ti)
        out[prec] = (np.array(d), np.array(T))
        torch.cuda.empty_cache()
    return out


def _welch(d32, d64):
    """Per-cell t statistic of the difference of the two means, its
    Welch-Satterthwaite degrees of freedom, and the cells where either side
    varies."""
    m = SEEDS
    v32, v64 = d32.var(0, ddof=1) / m, d64.var(0, ddof=1) / m
    se = np.sqrt(v32 + v64)
    live = se > 0
    t = np.zeros_like(se)
    t[live] = (d32.mean(0)[live] - d64.mean(0)[live]) / se[live]
    with np.errstate(invalid="ignore", divide="ignore"):
        nu = (v32 + v64) ** 2 / (v32 ** 2 / (m - 1) + v64 ** 2 / (m - 1))
    return t, np.where(live, nu, np.inf), live


@pytest.mark.parametrize("ti", range(len(TIMES)))
def test_fp32_density_within_3_standard_errors_of_fp64(runs, ti):
    from scipy import stats
    d32, d64 = runs["fp32"][0][:, ti], runs["fp64"][0][:, ti]
    t, nu, live = _welch(d32, d64)
    # cells where neither side ever varies hold the same value on both
    assert np.array_equal(d32.mean(0)[~live], d64.mean(0)[~live])
    K = int(live.sum())
    assert K > 300, K                      # the packet covers many blocks
    tl, nul = t[live], nu[live]
    # 3 standard errors: beyond it, cells at the rate the t-distribution gives
    p3 = 2 * stats.t.sf(3.0, nul)
    beyond = int((np.abs(tl) > 3.0).sum())
    mean_p, var_p = p3.sum(), (p3 * (1 - p3)).sum()
    assert beyond <= mean_p + 5 * math.sqrt(var_p) + 1, (beyond, mean_p, K)
    # no cell beyond the Bonferroni bound at family-wise level 1e-3
    bound = stats.t.isf(0.5e-3 / K, nul)
    assert np.all(np.abs(tl) < bound), (np.abs(tl).max(), bound.min())
    # the mean squared deviation (null: nu / (nu - 2) per cell)
    nul_c = np.maximum(nul, 4.5)
    e = nul_c / (nul_c - 2)
    v = 2 * nul_c ** 2 * (nul_c - 1) / ((nul_c - 2) ** 2 * (nul_c - 4))
    z = ((tl ** 2).sum() - e.sum()) / math.sqrt(v.sum())
    print("\ndensity t=%g: %d cells, %d beyond 3 SE (expected %.1f), max |t| %.2f "
          "(bound %.2f), mean t^2 %.3f (null %.3f, z %.2f)"
          % (TIMES[ti] * WL["dt"], K, beyond, mean_p, np.abs(tl).max(), bound.min(),
             (tl ** 2).mean(), e.mean(), z))
    assert z < 5.0, z


@pytest.mark.parametrize("ti", range(len(TIMES)))
def test_fp32_transmission_within_2e_3_of_fp64(runs, ti):
    T32, T64 = runs["fp32"][1][:, ti], runs["fp64"][1][:, ti]
    se = math.hypot(T32.std(ddof=1), T64.std(ddof=1)) / math.sqrt(SEEDS)
    print("\ntransmission t=%g: fp32 %.6f fp64 %.6f difference %.2e (combined SE %.2e)"
          % (TIMES[ti] * WL["dt"], T32.mean(), T64.mean(), T32.mean() - T64.mean(), se))
    assert se < 5e-4, se                   # resolution well inside the bound
    assert abs(T32.mean() - T64.mean()) <= 2e-3, (T32.mean(), T64.mean(), se)


def test_the_benchmark_size_matches_fp64(torch, runs):
    """1e8 particles, the benchmark's capacity (4 x 1e8 + 2^20) and graph
    replay, against the FP64 reference at both times."""
    d, T, live = _run(torch, "fp32", 100_000_000, 7, graphs=True)
    assert max(live) > 1.2e8                # the queues and arrays at full size
    d32s, T32s = runs["fp32"]
    d64, T64 = runs["fp64"]
    for ti in range(len(TIMES)):
        assert abs(T[ti] - T64[:, ti].mean()) <= 2e-3, (T[ti], T64[:, ti].mean())
        v = d32s[:, ti].var(0, ddof=1) / 10 + d64[:, ti].var(0, ddof=1) / SEEDS
        se = np.sqrt(v)
        live_c = se > 0
        z = (d[ti] - d64[:, ti].mean(0))[live_c] / se[live_c]
        K = int(live_c.sum())
        print("\n1e8 run t=%g: T %.6f (fp64 %.6f), %d cells, %d beyond 3 SE, max |z| %.2f, "
              "mean z^2 %.3f, live %d" % (TIMES[ti] * WL["dt"], T[ti], T64[:, ti].mean(), K,
                                          (np.abs(z) > 3).sum(), np.abs(z).max(),
                                          np.mean(z ** 2), live[ti]))
        assert (np.abs(z) > 3.0).sum() <= 0.01 * K + 5, ((np.abs(z) > 3).sum(), K)
        assert np.abs(z).max() < 7.0, np.abs(z).max()
        assert np.mean(z ** 2) < 1.5, np.mean(z ** 2)
