"""Oracle of the signed-particle Wigner branching random walk (arXiv:1709.02121).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
(``paper_1709_02121_gb300``) neither imports nor links anything here, and this
package imports nothing from it.

Contents
--------
* ``wbrw4_oracle.c`` -- the same for the 4D Helium-like system of Example 1
  (two electrons, soft-Coulomb kernels tabulated from Eq. 2, M = 3
  components); ``Oracle4`` below.
* ``wbrw_oracle.c`` -- plain FP64 C implementation of Alg. 1 (per interval),
  the signed histogram (Eq. signed_histogram), Alg. 3 and the signed residual
  bootstrap (Alg. 2 with Eq. lambda / double_bootstrap / boostrap_histogram),
  with its own Philox4x32-10.  Loaded here through ctypes.
* ``refs.py`` -- independent numerical references used to pin it: quadrature
  of the Wigner-kernel definition (Eq. 2), a split-step solver of the
  Schroedinger equation and a deterministic grid solver of the truncated Wigner
  equation (Eq. 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wbrw_oracle.c")
_SRC4 = os.path.join(_HERE, "wbrw4_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libwbrw_oracle.so")

SP1 = 1
SP2 = 2
WP = 3

# counter word 2 of the reserved streams (documented in wbrw_oracle.c)
STEP_INIT = 0xFFFFFFFF
STEP_REGEN = 0xFFFFFFFE
STEP_BOOT = 0xFFFFFFFD
STEP_ROUND = 0xFFFFFFFC

LEDGER = ("events", "kill_plus", "kill_minus", "out_plus", "out_minus",
          "particle_steps", "candidates", "first_pairs")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC4))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, _SRC4, "-lm"]
    # with OpenMP where the compiler has it (threads never change a result);
    # without it the oracle runs its chunks one after the other
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
    if r.returncode:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def max_threads() -> int:
    """Threads the oracle can use (1 if it was built without OpenMP)."""
    return int(lib().orc_max_threads())


class _Comp(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("om", ctypes.c_double),
                ("ph", ctypes.c_double), ("w", ctypes.c_double), ("xc", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [("hbar", ctypes.c_double), ("mass", ctypes.c_double),
                ("dt", ctypes.c_double), ("gamma0", ctypes.c_double),
                ("H", ctypes.c_double), ("w", ctypes.c_double),
                ("xc", ctypes.c_double),
                ("nx", ctypes.c_int), ("nk", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("kmin", ctypes.c_double), ("kmax", ctypes.c_double),
                ("strategy", ctypes.c_int),
                ("n_alpha", ctypes.c_longlong),
                ("seed", ctypes.c_ulonglong),
                ("instance", ctypes.c_int),
                ("tangent", ctypes.c_int), ("tquantum", ctypes.c_longlong),
                ("ncomp", ctypes.c_int), ("comp", _Comp * 4)]


EVENT_DTYPE = np.dtype([("pid", "<u8"), ("pid_plus", "<u8"),
                        ("pid_minus", "<u8"), ("step", "<u4"), ("j", "<u4"),
                        ("t", "<f8"), ("xe", "<f8"), ("kappa", "<f8"),
                        ("factor", "<f8"), ("kill_plus", "<i4"),
                        ("kill_minus", "<i4")])

EVENT4_DTYPE = np.dtype([("pid", "<u8"), ("pid_plus", "<u8"),
                         ("pid_minus", "<u8"), ("step", "<u4"), ("j", "<u4"),
                         ("t", "<f8"), ("xe", "<f8"), ("kappa", "<f8"),
                         ("factor", "<f8"), ("kill_plus", "<i4"),
                         ("kill_minus", "<i4"), ("xe2", "<f8"), ("comp", "<i4"),
                         ("pad", "<i4")])


class _Config4(ctypes.Structure):
    _fields_ = [("hbar", ctypes.c_double), ("mass", ctypes.c_double),
                ("dt", ctypes.c_double), ("Z", ctypes.c_double),
                ("a", ctypes.c_double), ("xc", ctypes.c_double),
                ("lam", ctypes.c_double), ("nx", ctypes.c_int), ("nk", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("kmin", ctypes.c_double), ("kmax", ctypes.c_double),
                ("ny", ctypes.c_int), ("nkap", ctypes.c_int),
                ("n_alpha", ctypes.c_longlong), ("seed", ctypes.c_ulonglong)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        D = ctypes.c_double
        LL = ctypes.c_longlong
        U32 = ctypes.c_uint32
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_u53.argtypes = [U32, U32]
        L.orc_u53.restype = D
        L.orc_vw_gauss.argtypes = [D] * 6
        L.orc_vw_gauss.restype = D
        L.orc_xi_gauss.argtypes = [D] * 5
        L.orc_xi_gauss.restype = D
        L.orc_create.argtypes = [ctypes.POINTER(_Config)]
        L.orc_create.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_cacc_ok.argtypes = [P]
        L.orc_gamma0.argtypes = [P]
        L.orc_gamma0.restype = D
        L.orc_enable_log.argtypes = [P, ctypes.c_int]
        L.orc_max_threads.argtypes = []
        L.orc_set_threads.argtypes = [P, ctypes.c_int]
        L.orc_threads.argtypes = [P]
        L.orc_init_gauss.argtypes = [P, LL, D, D, D]
        L.orc_set_particles.argtypes = [P, LL, P, P, P, P, LL]
        L.orc_step.argtypes = [P, ctypes.c_int]
        L.orc_annihilate.argtypes = [P]
        L.orc_histogram.argtypes = [P, P, P]
        L.orc_observables.argtypes = [P, P, P, P, P]
        L.orc_count.argtypes = [P]
        L.orc_count.restype = LL
        L.orc_step_index.argtypes = [P]
        L.orc_step_index.restype = LL
        L.orc_epoch.argtypes = [P]
        L.orc_epoch.restype = LL
        L.orc_get_particles.argtypes = [P, P, P, P, P]
        L.orc_get_grid.argtypes = [P, P]
        L.orc_set_grid.argtypes = [P, P, LL]
        L.orc_regenerate.argtypes = [P]
        L.orc_get_ledger.argtypes = [P, P]
        L.orc_get_wkill.argtypes = [P, P]
        L.orc_get_boot.argtypes = [P, P, P, P, P]
        L.orc_get_boot_counts.argtypes = [P, P, P]
        L.orc_log_count.argtypes = [P]
        L.orc_log_count.restype = LL
        L.orc_get_log.argtypes = [P, P]
        L.orc_event_size.restype = LL
        L.orc_event_outcome.argtypes = [P, ctypes.c_uint64, U32, U32, D,
                                        P, P, P]
        L.orc_get_tangent.argtypes = [P, P, P]
        L.orc_get_dgrid.argtypes = [P, P, P]
        L.orc_get_tkill.argtypes = [P, P]
        L.orc_tangent_transmission.argtypes = [P, P]
        assert L.orc_event_size() == EVENT_DTYPE.itemsize
        L.orc4_k0.argtypes = [D]
        L.orc4_k0.restype = D
        L.orc4_create.argtypes = [ctypes.POINTER(_Config4)]
        L.orc4_create.restype = P
        L.orc4_destroy.argtypes = [P]
        for name in ("orc4_gamma",):
            getattr(L, name).argtypes = [P, ctypes.c_int]
            getattr(L, name).restype = D
        L.orc4_Gamma.argtypes = [P]
        L.orc4_Gamma.restype = D
        L.orc4_enable_log.argtypes = [P, ctypes.c_int]
        L.orc4_get_table.argtypes = [P, ctypes.c_int, P, P, P]
        L.orc4_init_gauss.argtypes = [P, LL, D, D, D, D, D]
        L.orc4_event_outcome.argtypes = [P, ctypes.c_uint64, U32, U32, D, D, P, P, P, P]
        L.orc4_step.argtypes = [P, ctypes.c_int]
        L.orc4_annihilate.argtypes = [P]
        L.orc4_count.argtypes = [P]
        L.orc4_count.restype = LL
        L.orc4_epoch.argtypes = [P]
        L.orc4_epoch.restype = LL
        L.orc4_get_particles.argtypes = [P, P, P, P, P, P, P]
        L.orc4_get_grid.argtypes = [P, P]
        L.orc4_get_ledger.argtypes = [P, P]
        L.orc4_log_count.argtypes = [P]
        L.orc4_log_count.restype = LL
        L.orc4_get_log.argtypes = [P, P]
        L.orc4_event_size.restype = LL
        L.orc4_observables.argtypes = [P, P, P, P, P]
        assert L.orc4_event_size() == EVENT4_DTYPE.itemsize
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter (4 x uint32) under one key (2 x uint32)."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u53(a, b):
    return lib().orc_u53(int(a), int(b))


def vw_gauss(H, w, xc, hbar, x, kappa):
    return lib().orc_vw_gauss(H, w, xc, hbar, x, kappa)


def xi_gauss(H, w, xc, hbar, x):
    return lib().orc_xi_gauss(H, w, xc, hbar, x)


class Oracle:
    """One run of the FP64 oracle: a particle list plus its histogram state."""

    def __init__(self, *, hbar=1.0, mass=1.0, dt=0.1, gamma0=0.0, H=1.0,
                 w=1.0, xc=0.0, nx=240, nk=128, xmin=-60.0, xmax=60.0,
                 kmin=-6.4, kmax=6.4, strategy=SP1, n_alpha=200000, seed=0,
                 instance=0, tangent=False, tquantum=1.0, comps=(), threads=1):
        """comps: up to 4 dicts (a, b, om, ph, w, xc) of a time-dependent
        potential sum_m (a + b cos(om t + ph)) exp(-(x-xc)^2/(2 w^2)); when
        given, H, w, xc and gamma0 are not used.  threads: chunks of each
        interval, binning and regeneration run in parallel (results do not
        depend on it)."""
        cs = (_Comp * 4)(*[_Comp(c["a"], c["b"], c["om"], c["ph"], c["w"], c["xc"])
                           for c in comps])
        self.cfg = _Config(hbar, mass, dt, gamma0, H, w, xc, nx, nk, xmin,
                           xmax, kmin, kmax, strategy, n_alpha, seed, instance,
                           1 if tangent else 0, int(round(tquantum * 2.0 ** 32)),
                           len(comps), cs)
        self.nx, self.nk = nx, nk
        self.n_alpha = n_alpha
        self._s = lib().orc_create(ctypes.byref(self.cfg))
        if not self._s:
            raise ValueError("oracle rejected the configuration")
        if threads != 1 and lib().orc_set_threads(self._s, int(threads)):
            raise ValueError("threads must be >= 1")

    def __del__(self):
        s = getattr(self, "_s", None)
        if s and _lib is not None:
            _lib.orc_destroy(s)
            self._s = None

    @property
    def threads(self):
        return lib().orc_threads(self._s)

    # ---- set-up ---------------------------------------------------------
    @property
    def gamma0(self):
        return lib().orc_gamma0(self._s)

    def enable_log(self, on=True):
        lib().orc_enable_log(self._s, 1 if on else 0)

    def init_gauss(self, n, x0, sigma_x, k0):
        if lib().orc_init_gauss(self._s, n, x0, sigma_x, k0):
            raise MemoryError

    def set_particles(self, x, k, w, pid, step=0):
        x = np.ascontiguousarray(x, np.float64)
        k = np.ascontiguousarray(k, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        pid = np.ascontiguousarray(pid, np.uint64)
        if lib().orc_set_particles(self._s, len(x), _ptr(x), _ptr(k), _ptr(w),
                                   _ptr(pid), step):
            raise MemoryError

    # ---- the method -----------------------------------------------------
    def step(self, n=1):
        if lib().orc_step(self._s, n):
            raise MemoryError

    def annihilate(self):
        if lib().orc_annihilate(self._s):
            raise MemoryError

    def set_grid(self, grid, epoch):
        g = np.ascontiguousarray(grid, np.int32).reshape(-1)
        lib().orc_set_grid(self._s, _ptr(g), epoch)

    def regenerate(self):
        if lib().orc_regenerate(self._s):
            raise MemoryError

    # ---- read-out -------------------------------------------------------
    @property
    def n(self):
        return lib().orc_count(self._s)

    @property
    def step_index(self):
        return lib().orc_step_index(self._s)

    @property
    def epoch(self):
        return lib().orc_epoch(self._s)

    def particles(self):
        n = self.n
        x = np.empty(n)
        k = np.empty(n)
        w = np.empty(n)
        pid = np.empty(n, np.uint64)
        lib().orc_get_particles(self._s, _ptr(x), _ptr(k), _ptr(w), _ptr(pid))
        return x, k, w, pid

    def grid(self):
        g = np.empty(self.nx * self.nk, np.int32)
        lib().orc_get_grid(self._s, _ptr(g))
        return g.reshape(self.nx, self.nk)

    # ---- tangent mode (likelihood-ratio derivatives in H and w) -----------
    def tangent(self):
        """(tau_H, tau_w) of the current particles."""
        n = self.n
        tH, tw = np.empty(n), np.empty(n)
        lib().orc_get_tangent(self._s, _ptr(tH), _ptr(tw))
        return tH, tw

    def dgrid(self):
        """The tangent histogram (D_H, D_w) of the last resampling, 2^-32 units."""
        dH = np.empty(self.nx * self.nk, np.int64)
        dw = np.empty(self.nx * self.nk, np.int64)
        lib().orc_get_dgrid(self._s, _ptr(dH), _ptr(dw))
        return dH.reshape(self.nx, self.nk), dw.reshape(self.nx, self.nk)

    def tangent_killed(self):
        out = np.zeros(2)
        lib().orc_get_tkill(self._s, _ptr(out))
        return out

    def transmission_gradient(self):
        """(dT/dH, dT/dw) from the tangent histogram of the last resampling."""
        out = np.zeros(2)
        lib().orc_tangent_transmission(self._s, _ptr(out))
        return out

    def histogram(self):
        """Signed counts and FP64 weight sums of the current particles."""
        c = np.empty(self.nx * self.nk, np.int32)
        ws = np.empty(self.nx * self.nk, np.float64)
        lib().orc_histogram(self._s, _ptr(c), _ptr(ws))
        return c.reshape(self.nx, self.nk), ws.reshape(self.nx, self.nk)

    def observables(self, counts):
        c = np.ascontiguousarray(counts, np.int32).reshape(-1)
        dens = np.empty(self.nx * self.nk)
        marg = np.empty(self.nx)
        T = np.zeros(1)
        lib().orc_observables(self._s, _ptr(c), _ptr(dens), _ptr(marg),
                              _ptr(T))
        return dens.reshape(self.nx, self.nk), marg, float(T[0])

    def ledger(self):
        out = np.zeros(8, np.int64)
        lib().orc_get_ledger(self._s, _ptr(out))
        return dict(zip(LEDGER, out.tolist()))

    def killed_weight(self):
        out = np.zeros(2)
        lib().orc_get_wkill(self._s, _ptr(out))
        return out

    def boot_stats(self):
        n = np.zeros(2, np.int64)
        keep = np.zeros(2, np.int64)
        nr = np.zeros(2, np.int64)
        wfix = np.zeros(2, np.uint64)
        lib().orc_get_boot(self._s, _ptr(n), _ptr(keep), _ptr(nr), _ptr(wfix))
        return dict(n=n, keep=keep, nr=nr, wfix=wfix)

    def boot_counts(self):
        p = np.zeros(self.nx * self.nk, np.int64)
        m = np.zeros(self.nx * self.nk, np.int64)
        lib().orc_get_boot_counts(self._s, _ptr(p), _ptr(m))
        return p.reshape(self.nx, self.nk), m.reshape(self.nx, self.nk)

    def event_log(self):
        n = lib().orc_log_count(self._s)
        out = np.zeros(n, EVENT_DTYPE)
        if n:
            lib().orc_get_log(self._s, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def event_outcome(self, pid, step, j, xe):
        kap = ctypes.c_double()
        f = ctypes.c_double()
        gap = ctypes.c_double()
        emit = lib().orc_event_outcome(self._s, pid, step, j, xe,
                                       ctypes.byref(kap), ctypes.byref(f),
                                       ctypes.byref(gap))
        return bool(emit), kap.value, f.value, gap.value


def k0(z):
    """K0 of the 4D oracle (its integral representation, trapezoid rule)."""
    return lib().orc4_k0(float(z))


class Oracle4:
    """One run of the 4D Helium-like oracle (two electrons, M = 3 kernels)."""

    def __init__(self, *, hbar=1.0, mass=1.0, dt=0.02, Z=2.0, a=1.0, xc=0.0, lam=1.0,
                 nx=64, nk=64, xmin=-10.0, xmax=10.0, kmin=-6.4, kmax=6.4, ny=4096,
                 nkap=2048, n_alpha=100000, seed=0):
        self.cfg = _Config4(hbar, mass, dt, Z, a, xc, lam, nx, nk, xmin, xmax, kmin, kmax,
                            ny, nkap, n_alpha, seed)
        self.nx, self.nk, self.ny, self.nkap = nx, nk, ny, nkap
        self._s = lib().orc4_create(ctypes.byref(self.cfg))
        if not self._s:
            raise ValueError("oracle rejected the configuration")

    def __del__(self):
        s = getattr(self, "_s", None)
        if s and _lib is not None:
            _lib.orc4_destroy(s)
            self._s = None

    def gamma(self, t):
        return lib().orc4_gamma(self._s, t)

    @property
    def Gamma(self):
        return lib().orc4_Gamma(self._s)

    def table(self, t, with_S=False):
        A = np.empty(self.nkap)
        xi = np.empty(self.ny)
        S = np.empty((self.ny, self.nkap)) if with_S else None
        lib().orc4_get_table(self._s, t, _ptr(A), _ptr(xi), _ptr(S))
        return (A, xi, S) if with_S else (A, xi)

    def enable_log(self, on=True):
        lib().orc4_enable_log(self._s, 1 if on else 0)

    def init_gauss(self, n, x0, sigma_x, k0):
        if lib().orc4_init_gauss(self._s, n, x0[0], x0[1], sigma_x, k0[0], k0[1]):
            raise MemoryError

    def event_outcome(self, pid, step, j, x1e, x2e):
        comp = ctypes.c_int()
        kap, prob, gap = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        e = lib().orc4_event_outcome(self._s, pid, step, j, x1e, x2e, ctypes.byref(comp),
                                     ctypes.byref(kap), ctypes.byref(prob), ctypes.byref(gap))
        return bool(e), comp.value, kap.value, prob.value, gap.value

    def step(self, n=1):
        if lib().orc4_step(self._s, n):
            raise MemoryError

    def annihilate(self):
        if lib().orc4_annihilate(self._s):
            raise MemoryError

    @property
    def n(self):
        return lib().orc4_count(self._s)

    @property
    def epoch(self):
        return lib().orc4_epoch(self._s)

    def particles(self):
        n = self.n
        out = [np.empty(n) for _ in range(5)]
        pid = np.empty(n, np.uint64)
        lib().orc4_get_particles(self._s, *[_ptr(a) for a in out], _ptr(pid))
        x1, x2, k1, k2, w = out
        return x1, x2, k1, k2, w, pid

    def grid(self):
        g = np.empty(self.nx * self.nx * self.nk * self.nk, np.int32)
        lib().orc4_get_grid(self._s, _ptr(g))
        return g.reshape(self.nx, self.nx, self.nk, self.nk)

    def ledger(self):
        out = np.zeros(8, np.int64)
        lib().orc4_get_ledger(self._s, _ptr(out))
        return dict(zip(LEDGER, out.tolist()))

    def event_log(self):
        n = lib().orc4_log_count(self._s)
        out = np.zeros(n, EVENT4_DTYPE)
        if n:
            lib().orc4_get_log(self._s, _ptr(out))
        return out

    def observables(self, counts):
        c = np.ascontiguousarray(counts, np.int32).reshape(-1)
        f1 = np.empty(self.nx * self.nk)
        marg = np.empty(self.nx)
        right = np.zeros(1)
        lib().orc4_observables(self._s, _ptr(c), _ptr(f1), _ptr(marg), _ptr(right))
        return f1.reshape(self.nx, self.nk), marg, float(right[0])
