"""Seeded synthetic workloads of the signed-particle WBRW hot path.

Parameters only: this module holds none of the method's arithmetic and is
shared by the tests, the benchmark and the smoke check.  Every random number
the method draws comes from the counter-based stream keyed by ``seed`` that
each implementation computes itself.

The workloads take the structure of the paper's 2D experiments (Sec. 5: a
Gaussian wavepacket scattering on a Gaussian barrier, constant auxiliary rate
gamma0, resampling every T_A, N_alpha well above the histogram size) with
hbar = m = 1.  The paper's own runs use reference solutions and parameters
that are not available; these synthetic inputs stand in for them.
"""
from __future__ import annotations

# 2D Gaussian barrier, plain signed-particle WBRW (pair generation), FP64:
# V(x) = H exp(-x^2/(2 w^2)), H = w = 1; f0 = (1/pi) exp(-(x+15)^2/(2*2.5^2)
# - 2*2.5^2 (k-1.5)^2); 2e5 particles; dt = 0.1, 100 steps; 240 x 128 cells
# over x in [-60, 60), k in [-6.4, 6.4); resampling every 10 steps (T_A = 1).
GAUSS_2D_FP64_2E5 = dict(
    name="gauss2d_sp1_fp64_n2e5_240x128",
    H=1.0, w=1.0, xc=0.0, x0=-15.0, sigma_x=2.5, k0=1.5,
    n_alpha=200_000, dt=0.1, steps=100, resample_every=10,
    nx=240, nk=128, xmin=-60.0, xmax=60.0, kmin=-6.4, kmax=6.4,
    precision="fp64", strategy="sp1", seed=0, hbar=1.0, mass=1.0,
    gamma0=0.0,
)

# 2D Gaussian barrier at scale: 1e8 particles, FP32 state, FP64 observables;
# 1200 x 512 cells; dt = 0.05, 400 steps; resampling every 10 steps, by pair
# generation (sp1) or by the signed bootstrap filter (sp2).
GAUSS_2D_FP32_1E8 = dict(
    name="gauss2d_fp32_n1e8_1200x512",
    H=1.0, w=1.0, xc=0.0, x0=-15.0, sigma_x=2.5, k0=1.5,
    n_alpha=100_000_000, dt=0.05, steps=400, resample_every=10,
    nx=1200, nk=512, xmin=-60.0, xmax=60.0, kmin=-6.4, kmax=6.4,
    precision="fp32", strategy="sp1", seed=0, hbar=1.0, mass=1.0,
    gamma0=0.0,
)


def scaled(base: dict, **over) -> dict:
    """A copy of a workload with some fields replaced (smaller test cases)."""
    w = dict(base)
    w.update(over)
    return w


# A packet that meets the barrier within two time units: used to compare the
# method with the Schroedinger equation while the particle count stays small.
COLLISION_2D = dict(
    name="gauss2d_collision",
    H=1.0, w=1.0, xc=0.0, x0=-3.0, sigma_x=1.0, k0=1.5,
    n_alpha=20_000, dt=0.1, steps=20, resample_every=0,
    nx=160, nk=128, xmin=-20.0, xmax=20.0, kmin=-6.4, kmax=6.4,
    precision="fp64", strategy="sp1", seed=0, hbar=1.0, mass=1.0,
    gamma0=0.0,
)


# Batched 2D: 256 independent Gaussian-barrier problems in the same launches,
# FP32, 600 x 256 cells each over x in [-60, 60), k in [-6.4, 6.4), dt = 0.05,
# resampling every 10 intervals.  Per instance, drawn from a generator seeded
# with `seed`: H ~ U[0.5, 2], w ~ U[0.5, 2], k0 ~ U[1, 2.5] and an initial
# particle count (= N_alpha) log-uniform in [1e4, 4e6]; the packet is the one
# of the 2D workloads (x0 = -15, sigma_x = 2.5).
BATCH_2D_FP32_256 = dict(
    name="batch2d_fp32_256x600x256",
    instances=256, H_range=(0.5, 2.0), w_range=(0.5, 2.0), k0_range=(1.0, 2.5),
    n_range=(1e4, 4e6), x0=-15.0, sigma_x=2.5, xc=0.0,
    dt=0.05, resample_every=10,
    nx=600, nk=256, xmin=-60.0, xmax=60.0, kmin=-6.4, kmax=6.4,
    precision="fp32", strategy="sp1", seed=0, hbar=1.0, mass=1.0,
    gamma0=0.0, n_alpha=1, H=1.0, w=1.0, k0=1.5,
)


def batch_instances(spec: dict, n_scale: float = 1.0) -> list:
    """The seeded instance parameters of a batched workload (inputs only).
    n_scale shrinks every particle count (small test and profiling cases)."""
    import numpy as np
    rng = np.random.default_rng(spec["seed"])
    m = spec["instances"]
    H = rng.uniform(*spec["H_range"], m)
    w = rng.uniform(*spec["w_range"], m)
    k0 = rng.uniform(*spec["k0_range"], m)
    lo, hi = np.log(spec["n_range"][0]), np.log(spec["n_range"][1])
    n = np.exp(rng.uniform(lo, hi, m))
    out = []
    for i in range(m):
        cnt = max(1, int(round(n[i] * n_scale)))
        out.append(dict(H=float(H[i]), w=float(w[i]), xc=spec["xc"], x0=spec["x0"],
                        sigma_x=spec["sigma_x"], k0=float(k0[i]), n_init=cnt, n_alpha=cnt))
    return out


# 4D Helium-like system (two 1D electrons, Example 1 of the paper with
# soft-Coulomb terms): V = -Z/sqrt(x1^2+a^2) - Z/sqrt(x2^2+a^2)
# + 1/sqrt((x1-x2)^2+a^2), Z = 2, a = 1; kernels tabulated on 4096 y nodes x
# 2048 kappa cells; initial product of Gaussian packets with sigma = 1 at
# x0 = (-1, 1), k0 = (0.5, -0.5); 5e7 particles; 64^4 cells over
# x in [-10, 10)^2, k in [-6.4, 6.4)^2; dt = 0.02, 250 steps, resampling every
# 10 steps; FP32.
HE_4D_FP32_5E7 = dict(
    name="he4d_fp32_n5e7_64x64x64x64",
    dim=4, Z=2.0, a=1.0, lam=1.0, xc=0.0, ny=4096, nkap=2048,
    x0=(-1.0, 1.0), sigma_x=1.0, k0=(0.5, -0.5),
    n_alpha=50_000_000, dt=0.02, steps=250, resample_every=10,
    nx=64, nk=64, xmin=-10.0, xmax=10.0, kmin=-6.4, kmax=6.4,
    precision="fp32", strategy="sp1", seed=0, hbar=1.0, mass=1.0,
    gamma0=0.0, H=2.0, w=1.0,
)


# Differentiation, batched: the transmission T(H, w) of the 2D Gaussian
# barrier at t = 20 and its likelihood-ratio derivatives, at 64 parameter
# points (an 8 x 8 grid over H in [0.5, 2], w in [0.5, 2]) with 1e7
# particles each; FP32 particles with FP64 tangent weights; resampling (and
# the checkpoint of the state) every 16 intervals of 0.025 (0.05 would let
# the particle count grow about 8-fold between resamplings at H = 2); the
# packet and the 240 x 128 grid of the 2D workloads.
GRAD_2D_FP32_64 = dict(
    name="grad2d_fp32_64x1e7_240x128",
    H_points=(0.5, 2.0, 8), w_points=(0.5, 2.0, 8), n_per_point=10_000_000,
    H=1.0, w=1.0, xc=0.0, x0=-15.0, sigma_x=2.5, k0=1.5,
    n_alpha=10_000_000, dt=0.025, steps=800, resample_every=16,
    nx=240, nk=128, xmin=-60.0, xmax=60.0, kmin=-6.4, kmax=6.4,
    precision="fp32", strategy="sp1", seed=0, hbar=1.0, mass=1.0,
    gamma0=0.0, tangent=True, tquantum=1.0,
)


def grad_points(spec: dict) -> list:
    """The (H, w) parameter points of a differentiation workload, H-major."""
    import numpy as np
    Hs = np.linspace(*spec["H_points"])
    ws = np.linspace(*spec["w_points"])
    return [(float(h), float(v)) for h in Hs for v in ws]


# 2D scattering on the time-dependent double barrier of the paper's Sec. 5
# (Eq. tDV) with the switch on the left, as its text describes:
# V(x, t) = 0.8 (0.5 + 0.5 cos(pi + 0.1 t)) exp(-(x+10)^2/8)
#         + 0.8 exp(-(x-10)^2/8);
# the packet, grid and sizes of the 1e8 2D workload, 1200 intervals of 0.05
# (t = 60), resampling every 10.
TDV_2D_FP32_1E8 = dict(
    GAUSS_2D_FP32_1E8, name="tdv2d_fp32_n1e8_1200x512", steps=1200,
    comps=(dict(a=0.4, b=0.4, om=0.1, ph=3.141592653589793, w=2.0, xc=-10.0),
           dict(a=0.8, b=0.0, om=0.0, ph=0.0, w=2.0, xc=10.0)),
)
