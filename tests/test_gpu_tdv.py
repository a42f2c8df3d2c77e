"""GPU parity with a time-dependent potential (Remark 1, Eq. tDV).

FP64: the component choice, the heights at the event's absolute time and
the acceptance follow the oracle's operation order, so ids, event logs,
ledgers and cell counts agree exactly and positions to 1e-12.  A single
static component is the static run bit for bit.  FP32 agrees with the
time-dependent Schroedinger equation within Monte Carlo error.
"""
import numpy as np
import pytest

import workloads
from helpers import make_oracle
from oracle import refs

pytestmark = pytest.mark.gpu

REL = 1e-12
COMPS = [dict(a=0.5, b=0.5, om=3.0, ph=2.0, w=0.8, xc=-0.5),
         dict(a=0.7, b=0.0, om=0.0, ph=0.0, w=0.6, xc=1.2)]
WL = workloads.scaled(workloads.COLLISION_2D, n_alpha=4100, nx=100, nk=64, xmin=-25.0,
                      xmax=25.0, kmin=-3.2, kmax=3.2, resample_every=5, comps=tuple(COMPS))


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def sim_of(wl, capacity=600_000, event_log=0):
    from paper_1709_02121_gb300 import Simulation
    return Simulation(wl, capacity, event_log=event_log)


def oracle_of(wl, log=False):
    o = make_oracle(wl)
    o.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    if log:
        o.enable_log()
    return o


def close(a, b):
    return np.all(np.abs(a - b) <= REL * np.maximum(1.0, np.abs(b)))


def assert_same_particles(sim, o):
    x, k, s, w, pid = sim.particles()
    ox, ok_, ow, opid = o.particles()
    a, b = np.argsort(pid, kind="stable"), np.argsort(opid, kind="stable")
    assert np.array_equal(pid[a], opid[b])
    assert close(x[a], ox[b]) and close(k[a], ok_[b])
    assert np.array_equal(s[a].astype(np.float64), ow[b])


def test_steps_and_events_match_oracle():
    sim, o = sim_of(WL, event_log=200_000), oracle_of(WL, log=True)
    sim.step(13)          # into the second switching period of the first barrier
    o.step(13)
    assert_same_particles(sim, o)
    g, r = sim.event_log(), o.event_log()
    assert len(g) == len(r) and len(g) > 200
    kg = np.lexsort((g["j"], g["pid"], g["step"]))
    ko = np.lexsort((r["j"], r["pid"], r["step"]))
    for f in ("pid", "pid_plus", "pid_minus", "step", "j", "kill_plus", "kill_minus"):
        assert np.array_equal(g[kg][f], r[ko][f]), f
    for f in ("t", "xe", "kappa", "factor"):
        assert close(g[kg][f], r[ko][f]), f
    c, led = sim.counters(), o.ledger()
    for key in ("events", "kill_plus", "kill_minus", "particle_steps", "candidates",
                "first_pairs"):
        assert c[key] == led[key], key


def test_fused_schedule_matches_oracle():
    sim, o = sim_of(WL), oracle_of(WL)
    for period in range(4):
        sim.run(5)
        o.step(5)
        o.annihilate()
        assert np.array_equal(sim.grid_counts(), o.grid()), period
    dens, marg, T, live = sim.density()
    odens, omarg, oT = o.observables(o.grid())
    assert np.array_equal(dens, odens) and T == oT and live == o.n


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_static_component_is_the_static_run(precision):
    base = workloads.scaled(WL, precision=precision, comps=())
    one = workloads.scaled(WL, precision=precision,
                           comps=(dict(a=base["H"], b=0.0, om=0.0, ph=0.0, w=base["w"],
                                       xc=base["xc"]),))
    a, b = sim_of(base), sim_of(one)
    for _ in range(3):
        a.run(5)
        b.run(5)
        assert np.array_equal(a.grid_counts(), b.grid_counts())


def test_fp32_matches_the_time_dependent_schroedinger_equation():
    edges = np.linspace(-8.0, 8.0, 17)
    Vt = refs.gauss_components(COMPS)
    x, rho = refs.tdse_density_t(Vt, WL["x0"], WL["sigma_x"], WL["k0"], 2.0, L=80.0, n=4096,
                                 dt=2e-3)
    ref = refs.bin_density(x, rho, edges)
    cells = []
    n = 100_000
    for seed in range(10):
        wl = workloads.scaled(workloads.COLLISION_2D, precision="fp32", n_alpha=n, seed=seed,
                              comps=tuple(COMPS))
        sim = sim_of(wl, capacity=60 * n)
        sim.step(20)
        xs, ks, s, w, _ = sim.particles(with_pids=False)
        cells.append(np.histogram(xs, bins=edges, weights=w.astype(np.float64))[0] / n)
    cells = np.array(cells)
    m, se = cells.mean(0), cells.std(0, ddof=1) / np.sqrt(len(cells))
    z = (m - ref) / np.sqrt(se ** 2 + 1e-8)
    assert np.max(np.abs(z)) < 4.5, np.round(z, 2)
    assert np.mean(z ** 2) < 3.0, np.round(z, 2)
