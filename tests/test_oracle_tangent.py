"""Pins of the oracle's likelihood-ratio derivatives (tangent mode).

The paper has no differentiation; the tangent weights follow from the
first-moment measure of the branching process (the product of the birth
intensities V_W^+ along a lineage, Eq. 2) and are pinned here by:
  * exact identities: the signed particles are the plain run's, births add
    cancelling tangent pairs (so the total tangent changes only by the
    killed offspring's), and resampling carries every cell's tangent mass;
  * central finite differences of the same estimator with common random
    numbers (the rate gamma0 held fixed, so a change of H or w moves only
    acceptance decisions and kicks);
  * central finite differences of the transmission of the Schroedinger
    equation (split-step TDSE), which the method estimates.
"""
import numpy as np
import pytest

import workloads
from helpers import make_oracle
from oracle import refs

WL = workloads.scaled(workloads.COLLISION_2D, n_alpha=6000, gamma0=2.0)
# dT/dw vanishes near w = 1 for this packet (TDSE: -0.002); w = 0.5 gives -0.13
WLS = {"H": WL, "w": workloads.scaled(WL, w=0.5)}


def run(wl, steps, resample=0, **over):
    o = make_oracle(wl, **over)
    o.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    for s in range(steps):
        o.step(1)
        if resample and (s + 1) % resample == 0 and s + 1 < steps:
            o.annihilate()
    return o


def T_and_grad(o, n):
    x, k, w, _ = o.particles()
    tH, tw = o.tangent()
    right = x > 0
    return w[right].sum() / n, tH[right].sum() / n, tw[right].sum() / n


def test_signed_particles_are_those_of_the_plain_run():
    a = run(WL, 8, resample=4)
    b = run(WL, 8, resample=4, tangent=True)
    xa, ka, wa, pa = a.particles()
    xb, kb, wb, pb = b.particles()
    sel = wb != 0
    assert np.array_equal(pa, pb[sel]) and np.array_equal(xa, xb[sel])
    assert np.array_equal(ka, kb[sel]) and np.array_equal(wa, wb[sel])
    assert (~sel).sum() > 0   # tangent particles exist after the resampling


def test_births_add_cancelling_tangent_pairs():
    o = run(WL, 10, tangent=True)
    tH, tw = o.tangent()
    kill = o.tangent_killed()
    assert o.ledger()["events"] > 1000
    assert abs(tH.sum() + kill[0]) < 1e-9 * (np.abs(tH).sum() + 1)
    assert abs(tw.sum() + kill[1]) < 1e-9 * (np.abs(tw).sum() + 1)
    assert np.abs(tH).max() > 1.0


def test_resampling_carries_each_cells_tangent_mass():
    o = run(WL, 6, tangent=True, tquantum=0.5)
    x, k, w, pid = o.particles()
    tH, tw = o.tangent()
    o.annihilate()
    dH, dw = o.dgrid()
    # D is the fixed-point sum of the in-grid tangents
    dx = (WL["xmax"] - WL["xmin"]) / WL["nx"]
    dk = (WL["kmax"] - WL["kmin"]) / WL["nk"]
    ix = np.floor((x - WL["xmin"]) * (1 / dx)).astype(int)
    ik = np.floor((k - WL["kmin"]) * (1 / dk)).astype(int)
    ok = (ix >= 0) & (ix < WL["nx"]) & (ik >= 0) & (ik < WL["nk"])
    for t, d in ((tH, dH), (tw, dw)):
        ref = np.zeros((WL["nx"], WL["nk"]), np.int64)
        np.add.at(ref, (ix[ok], ik[ok]), np.rint(t[ok] * 2.0 ** 32).astype(np.int64))
        assert np.array_equal(ref, d)
    # the regenerated set: signed particles with tau = 0, and sign-0
    # particles that split each cell's D exactly, none above the quantum
    y, q, w2, pid2 = o.particles()
    sH, sw = o.tangent()
    assert np.all(sH[w2 != 0] == 0) and np.all(sw[w2 != 0] == 0)
    t0 = w2 == 0
    assert np.all(np.maximum(np.abs(sH[t0]), np.abs(sw[t0])) <= 0.5 + 1e-12)
    jx = np.floor((y[t0] - WL["xmin"]) * (1 / dx)).astype(int)
    jk = np.floor((q[t0] - WL["kmin"]) * (1 / dk)).astype(int)
    for t, d in ((sH[t0], dH), (sw[t0], dw)):
        back = np.zeros((WL["nx"], WL["nk"]))
        np.add.at(back, (jx, jk), t)
        assert np.allclose(back, d * 2.0 ** -32, rtol=1e-12, atol=1e-15)
    assert np.all(pid2[t0] & np.uint64(0x80000000))


def _lr_vs_fd(param, delta, steps, resample, nseed=12):
    wl = WLS[param]
    lr, fd = [], []
    for seed in range(nseed):
        o = run(wl, steps, resample=resample, tangent=True, seed=seed)
        T, gH, gw = T_and_grad(o, wl["n_alpha"])
        lr.append(gH if param == "H" else gw)
        Tp = T_and_grad(run(wl, steps, resample=resample, seed=seed,
                            **{param: wl[param] + delta}), wl["n_alpha"])[0]
        Tm = T_and_grad(run(wl, steps, resample=resample, seed=seed,
                            **{param: wl[param] - delta}), wl["n_alpha"])[0]
        fd.append((Tp - Tm) / (2 * delta))
    lr, fd = np.array(lr), np.array(fd)
    return lr.mean(), lr.std(ddof=1) / np.sqrt(nseed), fd.mean(), fd.std(ddof=1) / np.sqrt(nseed)


@pytest.mark.parametrize("param, delta", [("H", 0.05), ("w", 0.05)])
@pytest.mark.parametrize("resample", [0, 5])
def test_lr_agrees_with_finite_differences_under_common_random_numbers(param, delta, resample):
    m_lr, se_lr, m_fd, se_fd = _lr_vs_fd(param, delta, 20, resample)
    assert abs(m_lr) > 3 * se_lr                       # a derivative well above the noise
    assert abs(m_lr - m_fd) < 4.0 * np.hypot(se_lr, se_fd) + 0.01 * abs(m_fd), \
        (m_lr, se_lr, m_fd, se_fd)


@pytest.mark.parametrize("param", ["H", "w"])
def test_lr_agrees_with_the_schroedinger_equation(param):
    # dT/dtheta of the TDSE transmission at t = 2 by central differences
    def T_tdse(H, w):
        V = refs.gauss_potential(H, w, WL["xc"])
        x, rho = refs.tdse_density(V, WL["x0"], WL["sigma_x"], WL["k0"], 2.0, L=80.0, n=4096,
                                   dt=2e-3)
        return refs.bin_density(x, rho, np.array([0.0, 40.0 - 1e-9]))[0]
    wl = WLS[param]
    d = 1e-3
    hp = dict(H=wl["H"], w=wl["w"])
    hm = dict(hp)
    hp[param] += d
    hm[param] -= d
    ref = (T_tdse(**hp) - T_tdse(**hm)) / (2 * d)
    vals = []
    for seed in range(16):
        o = run(workloads.scaled(wl, n_alpha=20000), 20, tangent=True, seed=seed)
        T, gH, gw = T_and_grad(o, 20000)
        vals.append(gH if param == "H" else gw)
    vals = np.array(vals)
    m, se = vals.mean(), vals.std(ddof=1) / np.sqrt(len(vals))
    assert abs(m - ref) < 4.0 * se + 0.02 * abs(ref), (m, se, ref)
