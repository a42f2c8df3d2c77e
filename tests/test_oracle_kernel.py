"""Pins of the oracle's Wigner kernel V_W and pair-creation rate xi(x).

The closed form in the oracle is a reading derived from the definition of
V_W (Eq. 2) for a potential symmetric about x_c.  It is checked against
quadrature of the definition itself, against the symmetries and moments the
definition implies, and against the rate printed in Sec. 5.5.
"""
import json
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import refs

GOLD = os.path.join(os.path.dirname(__file__), "golden")

POTS = [(1.0, 1.0, 0.0), (0.6, 2.0, 30.0), (-0.8, 0.5, 1.5)]


@pytest.mark.parametrize("H,w,xc", POTS)
def test_vw_matches_quadrature_of_definition(oracle_mod, H, w, xc):
    V = refs.gauss_potential(H, w, xc)
    for dx in (-2.7, -0.4, 0.05, 0.8, 3.1):
        for kap in (-2.2, -0.6, 0.3, 0.9, 1.7):
            x = xc + dx
            closed = oracle_mod.vw_gauss(H, w, xc, 1.0, x, kap)
            quad = refs.vw_quadrature(V, x, kap)
            assert abs(closed - quad) <= 1e-9 * max(1.0, abs(quad)), (x, kap)


def test_vw_hbar_scaling(oracle_mod):
    V = refs.gauss_potential(0.6, 2.0, 30.0)
    for hbar in (0.5, 0.6582119569):
        a = oracle_mod.vw_gauss(0.6, 2.0, 30.0, hbar, 31.0, 0.4)
        b = refs.vw_quadrature(V, 31.0, 0.4, hbar=hbar)
        assert abs(a - b) < 1e-9 * abs(b)


def test_vw_antisymmetries(oracle_mod):
    H, w, xc = 1.3, 0.7, 2.0
    for x in (-1.0, 1.9, 2.5, 7.0):
        for kap in (0.2, 1.1, 3.0):
            v = oracle_mod.vw_gauss(H, w, xc, 1.0, x, kap)
            assert oracle_mod.vw_gauss(H, w, xc, 1.0, x, -kap) == -v
            mirrored = oracle_mod.vw_gauss(H, w, xc, 1.0, 2 * xc - x, kap)
            assert abs(mirrored + v) < 1e-14 * max(1, abs(v))


def test_vw_positive_and_negative_parts_balance(oracle_mod):
    # int V_W^+ dk = int V_W^- dk (Eq. def.xi_m): both equal xi(x)
    H, w, xc = 1.0, 1.0, 0.0
    for x in (0.3, 1.0, 2.5):
        f = lambda k: oracle_mod.vw_gauss(H, w, xc, 1.0, x, k)
        plus = integrate.quad(lambda k: max(f(k), 0.0), -10, 10, limit=4000)[0]
        minus = integrate.quad(lambda k: max(-f(k), 0.0), -10, 10, limit=4000)[0]
        assert abs(plus - minus) < 1e-8
        assert abs(plus - oracle_mod.xi_gauss(H, w, xc, 1.0, x)) < 1e-7


def test_vw_first_moment_is_the_classical_force(oracle_mod):
    # Theta_V[f] -> (1/hbar) V'(x) d_k f in the classical limit, i.e.
    # -int kappa V_W(x, kappa) dkappa = V'(x) / hbar for the kernel of Eq. 2
    H, w, xc = 0.9, 1.2, 0.4
    for x in (-0.7, 0.4, 1.0, 2.2):
        m1 = integrate.quad(lambda k: k * oracle_mod.vw_gauss(H, w, xc, 1.0, x, k),
                            -12, 12, limit=4000)[0]
        dV = -H * (x - xc) / (w * w) * np.exp(-((x - xc) ** 2) / (2 * w * w))
        assert abs(-m1 - dV) < 1e-9


def test_xi_closed_form_against_quadrature(oracle_mod):
    H, w, xc = 1.0, 1.0, 0.0
    for x in (1e-7, 1e-3, 0.05, 0.3, 0.7, 1.5, 4.0):
        q = integrate.quad(lambda k: 0.5 * abs(oracle_mod.vw_gauss(H, w, xc, 1.0, x, k)),
                           -12, 12, limit=8000, epsabs=1e-13)[0]
        assert abs(oracle_mod.xi_gauss(H, w, xc, 1.0, x) - q) < 2e-9


def test_xi_special_values(oracle_mod):
    # xi vanishes on the symmetry axis and tends to 2|H|/(pi hbar) far from it
    assert oracle_mod.xi_gauss(1.0, 1.0, 0.0, 1.0, 0.0) == 0.0
    far = oracle_mod.xi_gauss(1.0, 1.0, 0.0, 1.0, 40.0)
    assert abs(far - 2.0 / np.pi) < 1e-15
    xs = np.linspace(0, 5, 60)
    vals = [oracle_mod.xi_gauss(1.0, 1.0, 0.0, 1.0, x) for x in xs]
    assert np.all(np.diff(vals) >= -1e-15)  # monotone in |x - xc|
    assert oracle_mod.xi_gauss(-2.0, 1.0, 0.0, 1.0, 40.0) == pytest.approx(4 / np.pi)


def test_printed_rate_of_sec55(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "sec55_gamma.json")))
    xi_check = oracle_mod.xi_gauss(g["H_eV"], g["w"], 30.0, g["hbar_eV_fs"], 30.0 + 200.0)
    gamma = g["factor"] * xi_check
    assert abs(gamma - g["gamma_printed"]) < g["abs_tol"]
