"""Independent numerical references that pin the oracle.  TEST INFRASTRUCTURE.

Nothing here shares arithmetic with ``wbrw_oracle.c``: each function starts
from a definition in the paper (or from quantum mechanics the paper relies
on) and evaluates it by a different numerical route.

* ``vw_quadrature`` -- the Wigner kernel straight from its definition (Eq. 2),
  by Fourier quadrature of V(x+y/2) - V(x-y/2).
* ``tdse_density`` -- the Schroedinger equation whose Wigner transform is the
  Wigner equation (Eq. 1), by Strang split-step Fourier.  For a Gaussian
  wavepacket psi0 the Wigner function is the f0 used throughout.
* ``GridWigner`` -- a deterministic solver of the k-truncated Wigner equation
  (Eq. 1 with the nullification outside K of Sec. 2) on a phase-space grid:
  exact spectral shift in x for the free streaming, RK4 for Theta_V with the
  kernel V_W tabulated by quadrature on the k-differences.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate


def gauss_potential(H, w, xc):
    return lambda x: H * np.exp(-((np.asarray(x) - xc) ** 2) / (2.0 * w * w))


def vw_quadrature(V, x, kappa, hbar=1.0):
    """V_W(x, kappa) = 1/(i hbar 2 pi) int e^{-i kappa y} [V(x+y/2) - V(x-y/2)] dy.

    The bracket is odd in y, so the integral is -2i int_0^inf sin(kappa y) D(y)
    dy and V_W = -(1/(pi hbar)) int_0^inf sin(kappa y) D(y) dy.  Evaluated with
    QUADPACK's Fourier-integral rule (QAWF) for kappa != 0.
    """
    if kappa == 0.0:
        return 0.0
    D = lambda y: V(x + y / 2.0) - V(x - y / 2.0)
    sgn = 1.0
    if kappa < 0:
        kappa, sgn = -kappa, -1.0
    val, _ = integrate.quad(D, 0.0, np.inf, weight="sin", wvar=kappa,
                            limlst=200)
    return -sgn * val / (np.pi * hbar)


def gaussian_psi0(x, x0, sigma, k0):
    """psi0 = (2 pi sigma^2)^(-1/4) exp(-(x-x0)^2/(4 sigma^2) + i k0 x); its
    Wigner function is (1/pi) exp(-(x-x0)^2/(2 sigma^2) - 2 sigma^2 (k-k0)^2)."""
    return ((2 * np.pi * sigma ** 2) ** -0.25
            * np.exp(-((x - x0) ** 2) / (4 * sigma ** 2) + 1j * k0 * x))


def tdse_density(V, x0, sigma, k0, t, *, L=200.0, n=1 << 14, dt=1e-3,
                 hbar=1.0, mass=1.0):
    """|psi(x,t)|^2 on a periodic grid of n points over [-L/2, L/2)."""
    x = (np.arange(n) - n // 2) * (L / n)
    kx = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    psi = gaussian_psi0(x, x0, sigma, k0).astype(np.complex128)
    v = V(x)
    nsteps = int(round(t / dt))
    h = t / nsteps if nsteps else 0.0
    half_v = np.exp(-0.5j * v * h / hbar)
    kin = np.exp(-0.5j * hbar * kx ** 2 * h / mass)
    for _ in range(nsteps):
        psi = half_v * psi
        psi = np.fft.ifft(kin * np.fft.fft(psi))
        psi = half_v * psi
    return x, np.abs(psi) ** 2


def bin_density(x, rho, edges):
    """Integrate a fine-grid density over the cells given by edges."""
    dx = x[1] - x[0]
    cdf = np.concatenate([[0.0], np.cumsum(rho) * dx])
    xe = np.concatenate([x - dx / 2, [x[-1] + dx / 2]])
    return np.diff(np.interp(edges, xe, cdf))


class GridWigner:
    """Deterministic solver of the k-truncated Wigner equation on a grid.

    f lives on x_i (periodic, n_x points over [xa, xb)) and k_j (cell
    centres of K = [ka, kb), n_k points).  One step of length h is Strang
    split: half a free-streaming step (exact: spectral shift of each k-row by
    k h), one RK4 step of df/dt = Theta_V[f], half a free-streaming step.
    Theta_V[f](x, k_i) = sum_j W(x, k_i - k_j) f(x, k_j) with W the cell
    integral of V_W(x, .) over [q - dk/2, q + dk/2], q = k_i - k_j.  Values
    of Theta_V outside K never arise (the k grid is K), which is the
    nullification of Sec. 2.
    """

    def __init__(self, V, *, xa, xb, nx, ka, kb, nk, hbar=1.0, mass=1.0,
                 vw=None):
        self.x = xa + (np.arange(nx) + 0.0) * (xb - xa) / nx
        self.dx = (xb - xa) / nx
        self.dk = (kb - ka) / nk
        self.k = ka + (np.arange(nk) + 0.5) * self.dk
        self.hbar, self.mass = hbar, mass
        self.xi_freq = 2 * np.pi * np.fft.fftfreq(nx, d=self.dx)
        q = (np.arange(-(nk - 1), nk) * self.dk)
        # W[i, m] = int_{q_m - dk/2}^{q_m + dk/2} V_W(x_i, q) dq by Gauss-Legendre
        gx, gw = np.polynomial.legendre.leggauss(8)
        W = np.zeros((nx, len(q)))
        for a, b in zip(gx, gw):
            qq = q + 0.5 * self.dk * a
            W += 0.5 * self.dk * b * vw(self.x[:, None], qq[None, :])
        idx = np.arange(nk)[:, None] - np.arange(nk)[None, :] + (nk - 1)
        self.M = W[:, idx]  # (nx, nk, nk): M[x, i, j] = W(x, k_i - k_j)

    def theta(self, f):
        return np.matmul(self.M, f[:, :, None])[:, :, 0]

    def stream(self, f, h):
        fh = np.fft.fft(f, axis=0)
        phase = np.exp(-1j * self.xi_freq[:, None] * self.k[None, :]
                       * (self.hbar / self.mass) * h)
        return np.real(np.fft.ifft(fh * phase, axis=0))

    def run(self, f, t, h):
        n = int(round(t / h))
        h = t / n
        for _ in range(n):
            f = self.stream(f, h / 2)
            k1 = self.theta(f)
            k2 = self.theta(f + 0.5 * h * k1)
            k3 = self.theta(f + 0.5 * h * k2)
            k4 = self.theta(f + h * k3)
            f = f + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
            f = self.stream(f, h / 2)
        return f


def gauss_vw_closed(H, w, xc, hbar):
    """Vectorised closed form of V_W for the Gaussian barrier (the reading
    derived from Eq. 2), for building GridWigner tables."""
    def vw(x, q):
        vhat = H * w * np.sqrt(2 * np.pi) * np.exp(-2.0 * q * q * w * w)
        return (2.0 / (np.pi * hbar)) * vhat * np.sin(2.0 * (x - xc) * q)
    return vw


def wigner_gauss_f0(x, k, x0, sigma, k0):
    return (1.0 / np.pi) * np.exp(-((x - x0) ** 2) / (2 * sigma ** 2)
                                  - 2 * sigma ** 2 * (k - k0) ** 2)


def soft_coulomb_2e(Z, a, lam, xc=0.0):
    """V(x1, x2) of two electrons in 1D: -Z/sqrt((x_i-xc)^2+a^2) for each,
    plus lam/sqrt((x1-x2)^2+a^2)."""
    def V(x1, x2):
        return (-Z / np.sqrt((x1 - xc) ** 2 + a * a) - Z / np.sqrt((x2 - xc) ** 2 + a * a)
                + lam / np.sqrt((x1 - x2) ** 2 + a * a))
    return V


def tdse2_marginals(V, x0, sigma, k0, t, *, L=40.0, n=256, dt=2e-3, hbar=1.0, mass=1.0):
    """Two distinguishable particles in 1D: Strang split-step Fourier on an
    n x n periodic grid over [-L/2, L/2)^2 from the product of Gaussian
    wavepackets (x0[e], sigma, k0[e]).  Returns x and the position densities
    of particle 1 and particle 2 at time t."""
    x = (np.arange(n) - n // 2) * (L / n)
    kx = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    K1, K2 = np.meshgrid(kx, kx, indexing="ij")
    psi = np.outer(gaussian_psi0(x, x0[0], sigma, k0[0]),
                   gaussian_psi0(x, x0[1], sigma, k0[1])).astype(np.complex128)
    v = V(X1, X2)
    nsteps = int(round(t / dt))
    h = t / nsteps if nsteps else 0.0
    half_v = np.exp(-0.5j * v * h / hbar)
    kin = np.exp(-0.5j * hbar * (K1 ** 2 + K2 ** 2) * h / mass)
    for _ in range(nsteps):
        psi = half_v * psi
        psi = np.fft.ifft2(kin * np.fft.fft2(psi))
        psi = half_v * psi
    dens = np.abs(psi) ** 2
    dx = L / n
    return x, dens.sum(1) * dx, dens.sum(0) * dx


def gauss_components(comps):
    """V(x, t) = sum_m (a + b cos(om t + ph)) exp(-(x-xc)^2/(2 w^2))."""
    def V(x, t):
        x = np.asarray(x)
        out = np.zeros_like(x, dtype=np.float64)
        for c in comps:
            out = out + (c["a"] + c["b"] * np.cos(c["om"] * t + c["ph"])) * np.exp(
                -((x - c["xc"]) ** 2) / (2.0 * c["w"] ** 2))
        return out
    return V


def tdse_density_t(Vt, x0, sigma, k0, t, *, L=200.0, n=1 << 14, dt=1e-3, hbar=1.0, mass=1.0):
    """|psi(x,t)|^2 for a time-dependent potential Vt(x, t): Strang
    split-step Fourier with the potential of each step taken at its midpoint."""
    x = (np.arange(n) - n // 2) * (L / n)
    kx = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    psi = gaussian_psi0(x, x0, sigma, k0).astype(np.complex128)
    nsteps = int(round(t / dt))
    h = t / nsteps if nsteps else 0.0
    kin = np.exp(-0.5j * hbar * kx ** 2 * h / mass)
    for i in range(nsteps):
        half_v = np.exp(-0.5j * Vt(x, (i + 0.5) * h) * h / hbar)
        psi = half_v * psi
        psi = np.fft.ifft(kin * np.fft.fft(psi))
        psi = half_v * psi
    return x, np.abs(psi) ** 2
