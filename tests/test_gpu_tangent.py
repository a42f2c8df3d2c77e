"""GPU parity of the tangent mode (likelihood-ratio dT/dH, dT/dw).

FP64: the same tangent rules and the same operation order as the oracle's
tangent mode, so tangent weights agree to 1e-12 relative, the fixed-point
tangent histogram and therefore the gradients exactly, and the signed
particles are bit for bit those of the run without tangents.  FP32: the
gradient of the transmission against finite differences of the TDSE, with
the instances of a batch as independent replicas.
"""
import numpy as np
import pytest

import workloads
from helpers import make_oracle
from oracle import refs

pytestmark = pytest.mark.gpu

REL = 1e-12
WL = workloads.scaled(workloads.COLLISION_2D, n_alpha=4100, gamma0=2.0, nx=100, nk=64,
                      xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2, resample_every=5,
                      tangent=True, tquantum=0.5)


@pytest.fixture(scope="module", autouse=True)
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def sim_of(wl, capacity=800_000, **kw):
    from paper_1709_02121_gb300 import Simulation
    return Simulation(wl, capacity, **kw)


def oracle_of(wl):
    o = make_oracle(wl)
    o.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    return o


def close(a, b):
    return np.all(np.abs(a - b) <= REL * np.maximum(1.0, np.abs(b)))


def assert_same(sim, o):
    x, k, s, w, pid = sim.particles()
    tH, tw = sim.tangents()
    ox, ok_, ow, opid = o.particles()
    oH, ow_ = o.tangent()
    assert len(pid) == len(opid)
    a, b = np.argsort(pid, kind="stable"), np.argsort(opid, kind="stable")
    assert np.array_equal(pid[a], opid[b])
    assert close(x[a], ox[b]) and close(k[a], ok_[b])
    assert np.array_equal(s[a].astype(np.float64), ow[b])
    assert close(tH[a], oH[b]) and close(tw[a], ow_[b])
    return np.abs(tH).max()


def test_steps_carry_the_oracles_tangents():
    sim, o = sim_of(WL), oracle_of(WL)
    sim.step(7)
    o.step(7)
    assert assert_same(sim, o) > 1.0


def test_fused_schedule_gradients_match_the_oracle():
    sim, o = sim_of(WL), oracle_of(WL)
    for period in range(3):
        sim.run(5)
        o.step(5)
        o.annihilate()
        assert np.array_equal(sim.grid_counts(), o.grid()), period
        g = sim.transmission_gradients()
        assert np.array_equal(g, o.transmission_gradient()), (period, g, o.transmission_gradient())
    # the regenerated set, tangent particles included, then two more steps
    assert_same(sim, o)
    sim.run(2)
    o.step(2)
    assert_same(sim, o)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_signed_particles_are_those_of_the_plain_run(gpu, precision):
    a = sim_of(workloads.scaled(WL, precision=precision, tangent=False))
    b = sim_of(workloads.scaled(WL, precision=precision), stream=gpu.cuda.Stream())
    b.graph(True)
    for _ in range(4):
        a.run(5)
        b.run(5)
        assert np.array_equal(a.grid_counts(), b.grid_counts())
    assert a.counters()["events"] < b.counters()["events"]   # tangent particles branch too


def test_batch_instances_match_the_oracle():
    from paper_1709_02121_gb300 import Batch
    insts = [dict(H=1.0, w=1.0, x0=-3.0, sigma_x=1.0, k0=1.5, n_init=3000, n_alpha=3000,
                  gamma0=2.0),
             dict(H=1.6, w=0.6, x0=-4.0, sigma_x=1.2, k0=1.8, n_init=1200, n_alpha=1200,
                  gamma0=2.0)]
    b = Batch(WL, insts, 400_000)
    b.run(10)
    g = b.transmission_gradients()
    for i, v in enumerate(insts):
        o = make_oracle(WL, H=v["H"], w=v["w"], n_alpha=v["n_alpha"], instance=i)
        o.init_gauss(v["n_init"], v["x0"], v["sigma_x"], v["k0"])
        for _ in range(2):
            o.step(5)
            o.annihilate()
        assert np.array_equal(b.grid_counts()[i], o.grid())
        assert np.array_equal(g[i], o.transmission_gradient()), i


def test_fp32_gradient_matches_the_schroedinger_equation():
    # 24 instances of the same problem as independent replicas; t = 2 with
    # one resampling; dT/dH and dT/dw against central differences of the TDSE
    from paper_1709_02121_gb300 import Batch
    wl = workloads.scaled(workloads.COLLISION_2D, precision="fp32", gamma0=2.0, w=0.5,
                          resample_every=10, tangent=True)
    n = 40_000
    insts = [dict(H=1.0, w=0.5, x0=wl["x0"], sigma_x=wl["sigma_x"], k0=wl["k0"], n_init=n,
                  n_alpha=n, gamma0=2.0)] * 24
    b = Batch(wl, insts, 24 * n * 6)
    b.run(20)
    g = b.transmission_gradients()

    def T_tdse(H, w):
        V = refs.gauss_potential(H, w, 0.0)
        x, rho = refs.tdse_density(V, wl["x0"], wl["sigma_x"], wl["k0"], 2.0, L=80.0, n=4096,
                                   dt=2e-3)
        return refs.bin_density(x, rho, np.array([0.0, 40.0 - 1e-9]))[0]
    d = 1e-3
    ref = [(T_tdse(1.0 + d, 0.5) - T_tdse(1.0 - d, 0.5)) / (2 * d),
           (T_tdse(1.0, 0.5 + d) - T_tdse(1.0, 0.5 - d)) / (2 * d)]
    for c in range(2):
        m, se = g[:, c].mean(), g[:, c].std(ddof=1) / np.sqrt(len(g))
        assert abs(m - ref[c]) < 4.0 * se + 0.02 * abs(ref[c]), (c, m, se, ref[c])


@pytest.mark.parametrize("replay", [False, True])
def test_autograd_function_gives_the_tangent_runs_gradients(replay):
    """One pass (the forward runs in tangent mode) or replay (the backward
    reruns the forward in tangent mode): T is the run without tangents and
    the gradients those of a direct tangent run."""
    import torch
    from paper_1709_02121_gb300 import grad
    wl = workloads.scaled(workloads.COLLISION_2D, precision="fp32", n_alpha=20000,
                          gamma0=2.0, resample_every=5)
    H = torch.tensor([1.0, 1.5], dtype=torch.float64, requires_grad=True)
    w = torch.tensor([0.5, 0.8], dtype=torch.float64, requires_grad=True)
    T = grad.transmission(H, w, wl, 10, 1_000_000, replay=replay)
    (T * torch.tensor([1.0, 2.0], dtype=torch.float64)).sum().backward()
    T2, g, _ = grad.run_batch(wl, [1.0, 1.5], [0.5, 0.8], 10, True, 1_000_000)
    T0, _, _ = grad.run_batch(wl, [1.0, 1.5], [0.5, 0.8], 10, False, 1_000_000)
    assert np.array_equal(T.detach().numpy(), T2) and np.array_equal(T2, T0)
    assert np.array_equal(H.grad.numpy(), np.array([1.0, 2.0]) * g[:, 0])
    assert np.array_equal(w.grad.numpy(), np.array([1.0, 2.0]) * g[:, 1])
    # without a gradient asked for, the forward pass runs no tangents
    with torch.no_grad():
        assert np.array_equal(grad.transmission(H, w, wl, 10, 1_000_000).numpy(), T0)


@pytest.mark.parametrize("param, theta, reps", [("H", (1.0, 1.0), 48), ("w", (1.0, 0.5), 192)])
def test_lr_gradient_agrees_with_crn_central_differences(param, theta, reps):
    """FP64, central differences with delta = 1e-3 and common random numbers.

    Instance i of a batch draws from the streams of instance salt i whatever
    its parameters, so replica i at theta - delta, theta and theta + delta
    shares every random number (gamma0 is held at 2, so the candidate clock
    does not move either).  Per replica, FD_i = (T(theta + delta) -
    T(theta - delta)) / (2 delta) and the likelihood-ratio estimate LR_i of
    the same replica are both unbiased for dT/dtheta (FD up to delta^2), and
    their paired difference must average to zero within its standard error.
    A change of theta flips an acceptance decision with probability of order
    delta per event, so Var(FD_i) grows like 1/delta; resampling would re-key
    the particles of every cell after the first changed count (ids are
    slots in cell order) and break the common numbers, so the runs go to
    t = 2 without resampling and are binned once at the end.  A change of w
    moves every kick and so flips more decisions than a change of H: its
    differences are noisier per replica, and 192 replicas resolve them."""
    from paper_1709_02121_gb300 import Batch
    H, w = theta
    delta = 1e-3
    n = 40_000
    wl = workloads.scaled(workloads.COLLISION_2D, precision="fp64", gamma0=2.0, H=H, w=w,
                          resample_every=0, tangent=False)

    def batch(h, v, tangent):
        insts = [dict(H=h, w=v, x0=wl["x0"], sigma_x=wl["sigma_x"], k0=wl["k0"], n_init=n,
                      n_alpha=n, gamma0=2.0)] * reps
        b = Batch(dict(wl, tangent=tangent, tquantum=1.0), insts, reps * n * 16)
        b.run(20)
        b.annihilate()
        T = b.transmissions()
        g = b.transmission_gradients() if tangent else None
        b.close()
        return T, g

    sh = {"H": (delta, 0.0), "w": (0.0, delta)}[param]
    Tp, _ = batch(H + sh[0], w + sh[1], False)
    Tm, _ = batch(H - sh[0], w - sh[1], False)
    T0, g = batch(H, w, True)
    lr = g[:, 0 if param == "H" else 1]
    fd = (Tp - Tm) / (2 * delta)
    d = fd - lr
    se_d = d.std(ddof=1) / np.sqrt(reps)
    se_lr = lr.std(ddof=1) / np.sqrt(reps)
    print("\nd T/d%s: LR %.4f (SE %.4f), FD %.4f (SE %.4f), paired difference %.4f (SE %.4f)"
          % (param, lr.mean(), se_lr, fd.mean(), fd.std(ddof=1) / np.sqrt(reps), d.mean(),
             se_d))
    assert abs(lr.mean()) > 5 * se_lr                  # a derivative well above the noise
    assert abs(d.mean()) < 4.0 * se_d + 0.01 * abs(lr.mean()), (lr.mean(), fd.mean(), se_d)
