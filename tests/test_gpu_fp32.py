"""FP32 production path, checked in law: it draws its candidate clock as
geometric gaps between candidate intervals, so it is compared with the
Schroedinger equation and with the FP64 path (bit-identical to the oracle)
through estimates and their Monte Carlo standard errors."""
import math

import numpy as np
import pytest

import workloads
from oracle import refs

pytestmark = pytest.mark.gpu

WL = workloads.COLLISION_2D
EDGES = np.linspace(-8.0, 8.0, 17)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def tdse():
    V = refs.gauss_potential(WL["H"], WL["w"], WL["xc"])
    x, rho = refs.tdse_density(V, WL["x0"], WL["sigma_x"], WL["k0"], 2.0,
                               L=80.0, n=4096, dt=2e-3)
    cells = refs.bin_density(x, rho, EDGES)
    T = refs.bin_density(x, rho, np.array([0.0, 40.0 - 1e-9]))[0]
    return cells, T


def _gpu_estimates(precision, strategy, n, seeds, resample=0, steps=20, nx=160, nk=128):
    from paper_1709_02121_gb300 import Simulation
    cells, Ts = [], []
    for seed in seeds:
        wl = workloads.scaled(WL, precision=precision, strategy=strategy, n_alpha=n,
                              seed=seed, resample_every=resample, nx=nx, nk=nk)
        sim = Simulation(wl, capacity=40 * n)
        sim.run(steps)
        x, k, s, w, _ = sim.particles(with_pids=False)
        h, _ = np.histogram(x.astype(np.float64), bins=EDGES, weights=w.astype(np.float64))
        cells.append(h / n)
        Ts.append(np.sum(w[x > 0].astype(np.float64)) / n)
        sim.close()
    cells, Ts = np.array(cells), np.array(Ts)
    k = len(seeds)
    return cells.mean(0), cells.std(0, ddof=1) / np.sqrt(k), Ts.mean(), Ts.std(ddof=1) / np.sqrt(k)


@pytest.mark.parametrize("strategy,resample", [("sp1", 0), ("sp1", 5), ("sp2", 5)])
def test_fp32_matches_tdse(tdse, strategy, resample):
    ref, Tref = tdse
    m, se, T, Tse = _gpu_estimates("fp32", strategy, 400_000, range(4), resample=resample,
                                   nx=320, nk=256)
    z = (m - ref) / np.sqrt(se ** 2 + 1e-10)
    bias = 0.0 if resample == 0 else 2e-3
    assert np.max(np.abs(z) - bias / np.maximum(se, 1e-12)) < 4.5, np.round(z, 2)
    assert abs(T - Tref) < 2e-3 + 3 * Tse, (T, Tse, Tref)


def test_fp32_matches_fp64_path():
    m32, se32, T32, Tse32 = _gpu_estimates("fp32", "sp1", 400_000, range(4), resample=5)
    m64, se64, T64, Tse64 = _gpu_estimates("fp64", "sp1", 400_000, range(10, 14), resample=5)
    z = (m32 - m64) / np.sqrt(se32 ** 2 + se64 ** 2 + 1e-12)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert abs(T32 - T64) < 2e-3 + 3 * np.hypot(Tse32, Tse64)


@pytest.mark.parametrize("resample", [0, 5])
def test_fp32_candidate_tallies_follow_the_clock(resample):
    """A particle alive at the start of an interval has its first event in it
    with probability p = 1 - exp(-gamma0 dt) (Sec. 3.2), so the candidate
    intervals are Binomial(particle-steps, p) given the population.  Far from
    the barrier the acceptance |sin(2 x kappa)| averages 2/pi (Remark 3 with
    gamma0 = C/2), so the first events' pairs are Binomial(candidates, 2/pi).
    The packet at x0 = -15 stays beyond |x| = 5 for these 6 intervals."""
    from paper_1709_02121_gb300 import Simulation
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, precision="fp32", n_alpha=400_000,
                          resample_every=resample)
    sim = Simulation(wl, capacity=4_000_000)
    sim.run(6)
    c = sim.counters()
    sim.close()
    p = 1.0 - math.exp(-1.0 * wl["dt"])  # gamma0 = |H|/hbar = 1
    n = c["particle_steps"]
    z = (c["candidates"] - n * p) / math.sqrt(n * p * (1 - p))
    assert abs(z) < 4.5, (c["candidates"], n, z)
    q = 2.0 / math.pi
    z = (c["first_pairs"] - c["candidates"] * q) / math.sqrt(c["candidates"] * q * (1 - q))
    assert abs(z) < 4.5, (c["first_pairs"], c["candidates"], z)
    assert c["first_pairs"] <= c["events"]
