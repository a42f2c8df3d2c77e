"""Pins of the oracle's candidate-interval tallies (Sec. 3.2, Remark 3).

Under the constant auxiliary rate gamma0, a particle alive at the start of
an interval of length dt has its first event inside that interval with
probability p = 1 - exp(-gamma0 dt), independently across particles and
intervals given the population.  So the candidate intervals of a run are
Binomial(particle-steps, p).  With gamma0 = C/2 the acceptance of an event
is |sin(2 (x_e - x_c) kappa)|, kappa ~ N(0, sigma_kappa^2); far from the
barrier, where 2 |x_e - x_c| sigma_kappa >> 1, the phase is spread over many
periods and the mean acceptance is E|sin| = 2/pi (the ratio xi(inf)/gamma0).
With the bootstrap strategy every event emits a weighted pair.
"""
import math

import numpy as np

import workloads
from helpers import make_oracle, make_oracle4


def _binom_z(k, n, p):
    return (k - n * p) / math.sqrt(n * p * (1.0 - p))


def test_candidates_follow_the_clock_without_potential(oracle_mod):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, H=0.0, gamma0=1.0, n_alpha=4000)
    o = make_oracle(wl)
    o.init_gauss(4000, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(7)
    led = o.ledger()
    p = 1.0 - math.exp(-wl["gamma0"] * wl["dt"])
    assert led["particle_steps"] == 7 * 4000
    assert abs(_binom_z(led["candidates"], led["particle_steps"], p)) < 4.5
    # V = 0: no event is ever accepted
    assert led["first_pairs"] == 0 and led["events"] == 0


def test_first_events_accept_at_two_over_pi_far_from_the_barrier(oracle_mod):
    # the packet starts at x0 = -15 (sigma_x = 2.5) and moves at k0 = 1.5:
    # within 4 intervals of 0.1 it stays beyond |x| = 5, where the phase
    # 2 |x| kappa has a standard deviation above 5 rad
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=30_000)
    o = make_oracle(wl)
    o.init_gauss(30_000, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(4)
    led = o.ledger()
    p = 1.0 - math.exp(-o.gamma0 * wl["dt"])
    assert abs(_binom_z(led["candidates"], led["particle_steps"], p)) < 4.5
    assert abs(_binom_z(led["first_pairs"], led["candidates"], 2.0 / math.pi)) < 4.5
    assert led["first_pairs"] <= led["events"]


def test_bootstrap_strategy_pairs_every_first_event(oracle_mod):
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, strategy="sp2", n_alpha=5000)
    o = make_oracle(wl)
    o.init_gauss(5000, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(3)
    led = o.ledger()
    assert led["candidates"] > 1000
    assert led["first_pairs"] == led["candidates"]


def test_4d_candidates_follow_the_majorant_clock(oracle_mod):
    wl = workloads.scaled(workloads.HE_4D_FP32_5E7, precision="fp64", n_alpha=3000,
                          nx=16, nk=16)
    o = make_oracle4(wl)
    o.init_gauss(3000, wl["x0"], wl["sigma_x"], wl["k0"])
    o.step(8)
    led = o.ledger()
    p = 1.0 - math.exp(-o.Gamma * wl["dt"])
    assert led["candidates"] > 100
    assert abs(_binom_z(led["candidates"], led["particle_steps"], p)) < 4.5
    assert 0 < led["first_pairs"] <= min(led["candidates"], led["events"])
