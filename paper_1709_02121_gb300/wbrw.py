"""Python binding of the C ABI in include/wbrw.h (argument marshalling only).

The functions below carry the C names and forward to ``libwbrw.so`` through
ctypes; every step of the method runs in the library's CUDA kernels.  PyTorch
supplies device memory and the stream.  There is no CPU fallback: if the
library has not been built, loading it raises.

``Simulation`` bundles a context with the device buffers it needs.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwbrw.so")

OK, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_STATE, ERR_TIMEOUT, ERR_NUMERIC = 0, -1, -2, -3, -4, -5, -6
SP1_PAIR, SP2_BOOTSTRAP, WP = 1, 2, 3
FP64, FP32 = 0, 1
POT_GAUSSIAN, POT_SOFT_COULOMB_2E = 0, 1

# counter slots (WBRW_C_*)
COUNTERS = ("live", "events", "kill_plus", "kill_minus", "out_plus", "out_minus",
            "particle_steps", "log_len", "step", "epoch", "launches",
            "boot_nplus", "boot_nminus", "boot_nrplus", "boot_nrminus",
            "boot_wplus", "boot_wminus", "nonzero_cells", "error", "particle_steps_first",
            "candidates", "first_pairs")
C_COUNT = 24

SYMBOLS = ("wbrw_scratch_bytes", "wbrw_init", "wbrw_step", "wbrw_annihilate",
           "wbrw_run", "wbrw_density", "wbrw_particles", "wbrw_checkpoint",
           "wbrw_restore", "wbrw_profile", "wbrw_profile_read", "wbrw_profile_read_events",
           "wbrw_counters",
           "wbrw_sync_status", "wbrw_last_error", "wbrw_destroy",
           "wbrw_observables_static", "wbrw_batch_scratch_bytes", "wbrw_batch_init",
           "wbrw_instance_density", "wbrw_transmissions", "wbrw_particle_instances",
           "wbrw_graph", "wbrw_get_tuning", "wbrw_set_tuning", "wbrw_autotune",
           "wbrw_init4d", "wbrw_transmission_gradients", "wbrw_init_td",
           "wbrw_philox_chain", "wbrw_one_launch_periods")
TUNE_BPS_MAX, TUNE_PASSES_MAX = 4, 6
MAX_CAPACITY = 4293918720  # WBRW_MAX_CAPACITY: slots index in 32 bits
MAX_INSTANCES = 256


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("precision", ctypes.c_int),
                ("strategy", ctypes.c_int),
                ("hbar", ctypes.c_double), ("mass", ctypes.c_double),
                ("dt", ctypes.c_double), ("gamma0", ctypes.c_double),
                ("nx", ctypes.c_int), ("nk", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("kmin", ctypes.c_double), ("kmax", ctypes.c_double),
                ("resample_every", ctypes.c_int),
                ("n_alpha", ctypes.c_longlong),
                ("seed", ctypes.c_ulonglong),
                ("table_ny", ctypes.c_int), ("table_nkappa", ctypes.c_int),
                ("tangent", ctypes.c_int), ("tangent_quantum", ctypes.c_double)]


class Potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("H", ctypes.c_double),
                ("w", ctypes.c_double), ("xc", ctypes.c_double),
                ("ee", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("pot", Potential), ("x0", ctypes.c_double), ("sigma_x", ctypes.c_double),
                ("k0", ctypes.c_double), ("n_init", ctypes.c_longlong),
                ("n_alpha", ctypes.c_longlong), ("gamma0", ctypes.c_double)]


class Component(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("omega", ctypes.c_double),
                ("phase", ctypes.c_double), ("w", ctypes.c_double), ("xc", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int), ("event_passes", ctypes.c_int)]


class Buffers(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("k", ctypes.c_void_p),
                ("s", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("capacity", ctypes.c_longlong),
                ("grid", ctypes.c_void_p), ("grid_cells", ctypes.c_longlong),
                ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_size_t),
                ("event_log", ctypes.c_void_p),
                ("event_log_capacity", ctypes.c_longlong),
                ("tangent", ctypes.c_void_p)]


EVENT_DTYPE = np.dtype([("pid", "<u8"), ("pid_plus", "<u8"), ("pid_minus", "<u8"),
                        ("step", "<u4"), ("j", "<u4"), ("t", "<f8"), ("xe", "<f8"),
                        ("kappa", "<f8"), ("factor", "<f8"), ("kill_plus", "<i4"),
                        ("kill_minus", "<i4"), ("xe2", "<f8"), ("comp", "<i4"),
                        ("pad", "<i4")])

_lib = None


class WbrwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("wbrw status %d: %s" % (status, msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load libwbrw.so (built by paper_1709_02121_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libwbrw.so is not built (%s); run "
                           "paper_1709_02121_gb300.build.build() first" % path)
    L = ctypes.CDLL(path)
    P, LL, I = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
    L.wbrw_scratch_bytes.argtypes = [ctypes.POINTER(Config), LL]
    L.wbrw_scratch_bytes.restype = ctypes.c_size_t
    L.wbrw_init.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Potential),
                            ctypes.POINTER(Buffers), LL, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, P,
                            ctypes.POINTER(P)]
    L.wbrw_init4d.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Potential),
                              ctypes.POINTER(Buffers), LL, P, ctypes.c_double, P, P,
                              ctypes.POINTER(P)]
    L.wbrw_init4d.restype = I
    L.wbrw_init_td.argtypes = [ctypes.POINTER(Config), I, P, ctypes.POINTER(Buffers), LL,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, P,
                               ctypes.POINTER(P)]
    L.wbrw_init_td.restype = I
    L.wbrw_transmission_gradients.argtypes = [P, P]
    L.wbrw_transmission_gradients.restype = I
    L.wbrw_batch_scratch_bytes.argtypes = [ctypes.POINTER(Config), I, LL]
    L.wbrw_batch_scratch_bytes.restype = ctypes.c_size_t
    L.wbrw_batch_init.argtypes = [ctypes.POINTER(Config), I, ctypes.POINTER(Instance),
                                  ctypes.POINTER(Buffers), P, ctypes.POINTER(P)]
    L.wbrw_instance_density.argtypes = [P, I, P, P, P, P]
    L.wbrw_transmissions.argtypes = [P, P]
    L.wbrw_particle_instances.argtypes = [P, P]
    for name in ("wbrw_init", "wbrw_step", "wbrw_annihilate", "wbrw_run",
                 "wbrw_density", "wbrw_particles", "wbrw_checkpoint",
                 "wbrw_restore", "wbrw_profile", "wbrw_profile_read",
                 "wbrw_profile_read_events", "wbrw_counters", "wbrw_sync_status", "wbrw_batch_init",
                 "wbrw_instance_density", "wbrw_transmissions",
                 "wbrw_particle_instances", "wbrw_graph", "wbrw_get_tuning",
                 "wbrw_set_tuning", "wbrw_autotune"):
        getattr(L, name).restype = I
    L.wbrw_get_tuning.argtypes = [P, P]
    L.wbrw_set_tuning.argtypes = [P, P]
    L.wbrw_autotune.argtypes = [P, I, P, P]
    L.wbrw_graph.argtypes = [P, I]
    L.wbrw_one_launch_periods.argtypes = [P, I]
    L.wbrw_one_launch_periods.restype = I
    L.wbrw_checkpoint.argtypes = [P, P, P, P]
    L.wbrw_restore.argtypes = [P, P, LL, LL]
    L.wbrw_profile.argtypes = [P, I]
    L.wbrw_profile_read.argtypes = [P, P, P]
    L.wbrw_profile_read_events.argtypes = [P, P, P]
    L.wbrw_step.argtypes = [P, I]
    L.wbrw_annihilate.argtypes = [P]
    L.wbrw_run.argtypes = [P, I]
    L.wbrw_density.argtypes = [P, P, P, P, P]
    L.wbrw_particles.argtypes = [P, P, P]
    L.wbrw_counters.argtypes = [P, P]
    L.wbrw_sync_status.argtypes = [P]
    L.wbrw_last_error.argtypes = [P]
    L.wbrw_last_error.restype = ctypes.c_char_p
    L.wbrw_destroy.argtypes = [P]
    L.wbrw_destroy.restype = None
    D = ctypes.c_double
    L.wbrw_observables_static.argtypes = [P, I, I, D, D, D, D, LL, P, P, P, P]
    L.wbrw_observables_static.restype = I
    L.wbrw_philox_chain.argtypes = [ctypes.c_ulonglong, I, LL, P, P]
    L.wbrw_philox_chain.restype = I
    _lib = L
    return L


def _check(ctx, st):
    if st != OK:
        msg = load().wbrw_last_error(ctx).decode() if ctx else ""
        raise WbrwError(st, msg)


# ---- the C calls, same names ------------------------------------------------
def wbrw_scratch_bytes(cfg: Config, capacity: int) -> int:
    return load().wbrw_scratch_bytes(ctypes.byref(cfg), capacity)


def wbrw_init(cfg, pot, bufs, n_init, x0, sigma_x, k0, stream_ptr):
    ctx = ctypes.c_void_p()
    st = load().wbrw_init(ctypes.byref(cfg), ctypes.byref(pot), ctypes.byref(bufs),
                          n_init, x0, sigma_x, k0, ctypes.c_void_p(stream_ptr),
                          ctypes.byref(ctx))
    if st != OK:
        raise WbrwError(st, "wbrw_init rejected its arguments")
    return ctx


def wbrw_init4d(cfg, pot, bufs, n_init, x0, sigma_x, k0, stream_ptr):
    ctx = ctypes.c_void_p()
    x0a = (ctypes.c_double * 2)(*x0)
    k0a = (ctypes.c_double * 2)(*k0)
    st = load().wbrw_init4d(ctypes.byref(cfg), ctypes.byref(pot), ctypes.byref(bufs), n_init,
                            x0a, sigma_x, k0a, ctypes.c_void_p(stream_ptr), ctypes.byref(ctx))
    if st != OK:
        raise WbrwError(st, "wbrw_init4d rejected its arguments")
    return ctx


def wbrw_init_td(cfg, comps, bufs, n_init, x0, sigma_x, k0, stream_ptr):
    """comps: dicts with a, b, om, ph, w, xc (see include/wbrw.h)."""
    arr = (Component * len(comps))(*[Component(c["a"], c["b"], c["om"], c["ph"], c["w"],
                                               c["xc"]) for c in comps])
    ctx = ctypes.c_void_p()
    st = load().wbrw_init_td(ctypes.byref(cfg), len(comps), arr, ctypes.byref(bufs), n_init,
                             x0, sigma_x, k0, ctypes.c_void_p(stream_ptr), ctypes.byref(ctx))
    if st != OK:
        raise WbrwError(st, "wbrw_init_td rejected its arguments")
    return ctx


def wbrw_batch_scratch_bytes(cfg: Config, ninst: int, capacity: int) -> int:
    return load().wbrw_batch_scratch_bytes(ctypes.byref(cfg), ninst, capacity)


def wbrw_batch_init(cfg, instances, bufs, stream_ptr):
    arr = (Instance * len(instances))(*instances)
    ctx = ctypes.c_void_p()
    st = load().wbrw_batch_init(ctypes.byref(cfg), len(instances), arr, ctypes.byref(bufs),
                                ctypes.c_void_p(stream_ptr), ctypes.byref(ctx))
    if st != OK:
        raise WbrwError(st, "wbrw_batch_init rejected its arguments")
    return ctx


def wbrw_instance_density(ctx, inst, nx, nk):
    dens = np.empty(nx * nk, np.float64)
    marg = np.empty(nx, np.float64)
    T = ctypes.c_double()
    live = ctypes.c_longlong()
    _check(ctx, load().wbrw_instance_density(ctx, inst, dens.ctypes.data, marg.ctypes.data,
                                             ctypes.byref(T), ctypes.byref(live)))
    return dens.reshape(nx, nk), marg, T.value, live.value


def wbrw_transmissions(ctx, ninst):
    out = np.empty(ninst, np.float64)
    _check(ctx, load().wbrw_transmissions(ctx, out.ctypes.data))
    return out


def wbrw_particle_instances(ctx, inst_dev_ptr):
    _check(ctx, load().wbrw_particle_instances(ctx, ctypes.c_void_p(inst_dev_ptr)))


def wbrw_transmission_gradients(ctx, ninst):
    """(dT/dH, dT/dw) per instance, shape (ninst, 2)."""
    out = np.empty(2 * ninst, np.float64)
    _check(ctx, load().wbrw_transmission_gradients(ctx, out.ctypes.data))
    return out.reshape(ninst, 2)


def wbrw_step(ctx, nsteps):
    _check(ctx, load().wbrw_step(ctx, nsteps))


def wbrw_annihilate(ctx):
    _check(ctx, load().wbrw_annihilate(ctx))


def wbrw_run(ctx, nsteps):
    _check(ctx, load().wbrw_run(ctx, nsteps))


def wbrw_density(ctx, nx, nk, dens=None, marg=None):
    """(density, x-marginal, transmission, live particles) of the current
    histogram.  dens (nx*nk doubles) and marg (nx doubles) may be given as
    host arrays to write into, e.g. views of pinned memory, which the copies
    from the device reach at full speed; new arrays otherwise."""
    dens = np.empty(nx * nk, np.float64) if dens is None else dens.reshape(-1)
    marg = np.empty(nx, np.float64) if marg is None else marg.reshape(-1)
    if (dens.dtype != np.float64 or marg.dtype != np.float64 or dens.size != nx * nk
            or marg.size != nx or not dens.flags.c_contiguous or not marg.flags.c_contiguous):
        raise ValueError("density and marginal buffers must be contiguous float64 of nx*nk and nx")
    T = ctypes.c_double()
    live = ctypes.c_longlong()
    _check(ctx, load().wbrw_density(ctx, dens.ctypes.data, marg.ctypes.data,
                                    ctypes.byref(T), ctypes.byref(live)))
    return dens.reshape(nx, nk), marg, T.value, live.value


def wbrw_particles(ctx, pid_dev_ptr=None):
    n = ctypes.c_longlong()
    _check(ctx, load().wbrw_particles(ctx, ctypes.byref(n),
                                      ctypes.c_void_p(pid_dev_ptr) if pid_dev_ptr else None))
    return n.value


def wbrw_checkpoint(ctx, grid_out_ptr):
    step = ctypes.c_longlong()
    epoch = ctypes.c_longlong()
    _check(ctx, load().wbrw_checkpoint(ctx, ctypes.c_void_p(grid_out_ptr), ctypes.byref(step),
                                       ctypes.byref(epoch)))
    return step.value, epoch.value


def wbrw_restore(ctx, grid_ptr, step, epoch):
    _check(ctx, load().wbrw_restore(ctx, ctypes.c_void_p(grid_ptr), step, epoch))


def wbrw_graph(ctx, enable=True):
    _check(ctx, load().wbrw_graph(ctx, 1 if enable else 0))


def wbrw_one_launch_periods(ctx, enable=True):
    _check(ctx, load().wbrw_one_launch_periods(ctx, 1 if enable else 0))


def wbrw_get_tuning(ctx):
    t = Tuning()
    _check(ctx, load().wbrw_get_tuning(ctx, ctypes.byref(t)))
    return t.blocks_per_sm, t.event_passes


def wbrw_set_tuning(ctx, blocks_per_sm, event_passes):
    t = Tuning(blocks_per_sm, event_passes)
    _check(ctx, load().wbrw_set_tuning(ctx, ctypes.byref(t)))


def wbrw_autotune(ctx, trials=2):
    """Returns ((blocks_per_sm, event_passes), table) with table[b-1, p] the
    fastest period time in ms of that setting (negative: capacity limit)."""
    t = Tuning()
    table = np.zeros((TUNE_BPS_MAX, TUNE_PASSES_MAX + 1), np.float64)
    _check(ctx, load().wbrw_autotune(ctx, trials, ctypes.byref(t), table.ctypes.data))
    return (t.blocks_per_sm, t.event_passes), table


def wbrw_profile(ctx, enable=True):
    _check(ctx, load().wbrw_profile(ctx, 1 if enable else 0))


def wbrw_profile_read(ctx):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(ctx, load().wbrw_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def wbrw_profile_read_events(ctx):
    """(summed ms, launches) of the event kernel since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(ctx, load().wbrw_profile_read_events(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def wbrw_counters(ctx):
    out = np.zeros(C_COUNT, np.int64)
    _check(ctx, load().wbrw_counters(ctx, out.ctypes.data))
    return dict(zip(COUNTERS, out.tolist()))


def wbrw_sync_status(ctx):
    return load().wbrw_sync_status(ctx)


def wbrw_last_error(ctx):
    return load().wbrw_last_error(ctx).decode()


def wbrw_observables_static(grid_ptr, nx, nk, xmin, xmax, kmin, kmax, n_alpha,
                            density_ptr, marginal_ptr, transmission_ptr, stream_ptr):
    """Allocation-free observables of a device histogram (device outputs)."""
    return load().wbrw_observables_static(
        ctypes.c_void_p(grid_ptr), nx, nk, xmin, xmax, kmin, kmax, n_alpha,
        ctypes.c_void_p(density_ptr) if density_ptr else None,
        ctypes.c_void_p(marginal_ptr), ctypes.c_void_p(transmission_ptr),
        ctypes.c_void_p(stream_ptr))


def wbrw_philox_chain(seed, iters, nthreads, out_ptr, stream_ptr):
    """Launch the chained Philox rate probe (device output, async)."""
    return load().wbrw_philox_chain(seed, iters, nthreads, ctypes.c_void_p(out_ptr),
                                    ctypes.c_void_p(stream_ptr))


def wbrw_destroy(ctx):
    if ctx:
        load().wbrw_destroy(ctx)


# ---- convenience: a context plus its torch-owned buffers --------------------
class Simulation:
    """One WBRW run on the current CUDA device.

    ``wl`` is a workload dict (see workloads.py); ``capacity`` bounds the
    particles held at once (and each offspring wave).
    """

    ninst = 1

    def __init__(self, wl: dict, capacity: int, *, event_log: int = 0, stream=None):
        self._buffers(wl, capacity, event_log, stream)
        self.pot = Potential(POT_GAUSSIAN, wl["H"], wl["w"], wl["xc"])
        if wl.get("comps"):   # a time-dependent potential (sum of components)
            self.ctx = wbrw_init_td(self.cfg, list(wl["comps"]), self.bufs, int(wl["n_alpha"]),
                                    wl["x0"], wl["sigma_x"], wl["k0"], self.stream.cuda_stream)
        else:
            self.ctx = wbrw_init(self.cfg, self.pot, self.bufs, int(wl["n_alpha"]),
                                 wl["x0"], wl["sigma_x"], wl["k0"], self.stream.cuda_stream)

    def _buffers(self, wl, capacity, event_log, stream):
        import torch
        self.torch = torch
        self.wl = dict(wl)
        prec = FP64 if wl["precision"] == "fp64" else FP32
        strat = {"sp1": SP1_PAIR, "sp2": SP2_BOOTSTRAP, "wp": WP}[wl["strategy"]]
        self.dim = int(wl.get("dim", 2))
        self.cfg = Config(self.dim, prec, strat, wl["hbar"], wl["mass"], wl["dt"], wl["gamma0"],
                          wl["nx"], wl["nk"], wl["xmin"], wl["xmax"], wl["kmin"], wl["kmax"],
                          wl["resample_every"], int(wl["n_alpha"]), int(wl["seed"]),
                          int(wl.get("ny", 0)), int(wl.get("nkap", 0)),
                          1 if wl.get("tangent") else 0, float(wl.get("tquantum", 1.0)))
        dev = torch.device("cuda", torch.cuda.current_device())
        fdt = torch.float64 if prec == FP64 else torch.float32
        self.nx, self.nk = wl["nx"], wl["nk"]
        self.capacity = int(capacity)
        nd = 2 if self.dim == 4 else 1   # coordinates per particle
        self.x = torch.empty(nd * self.capacity, dtype=fdt, device=dev)
        self.k = torch.empty(nd * self.capacity, dtype=fdt, device=dev)
        self.s = torch.empty(self.capacity, dtype=torch.int8, device=dev)
        self.w = torch.empty(self.capacity, dtype=fdt, device=dev) if strat != SP1_PAIR else None
        self.tan = (torch.zeros(2 * self.capacity, dtype=torch.float64, device=dev)
                    if wl.get("tangent") else None)
        self.cells = (self.nx * self.nx * self.nk * self.nk if self.dim == 4
                      else self.nx * self.nk)
        cells = self.ninst * self.cells
        self.grid = torch.zeros(cells, dtype=torch.int32, device=dev)
        nbytes = (wbrw_batch_scratch_bytes(self.cfg, self.ninst, self.capacity)
                  if isinstance(self, Batch) else wbrw_scratch_bytes(self.cfg, self.capacity))
        if nbytes == 0:
            raise ValueError("invalid configuration")
        self.scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.log = (torch.zeros(event_log * EVENT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
                    if event_log else None)
        self.bufs = Buffers(self.x.data_ptr(), self.k.data_ptr(), self.s.data_ptr(),
                            self.w.data_ptr() if self.w is not None else None,
                            self.capacity, self.grid.data_ptr(), cells,
                            self.scratch.data_ptr(), nbytes,
                            self.log.data_ptr() if self.log is not None else None,
                            event_log, self.tan.data_ptr() if self.tan is not None else None)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        # the buffers were made on torch's current stream: the context's
        # stream must see them finished
        self.stream.wait_stream(torch.cuda.current_stream())

    def step(self, n=1):
        wbrw_step(self.ctx, n)

    def annihilate(self):
        wbrw_annihilate(self.ctx)

    def run(self, n):
        wbrw_run(self.ctx, n)

    def autotune(self, trials=2):
        """Time the next resampling period under every launch shape and keep
        the fastest (results do not depend on it)."""
        return wbrw_autotune(self.ctx, trials)

    def tuning(self, blocks_per_sm=None, event_passes=None):
        b, p = wbrw_get_tuning(self.ctx)
        if blocks_per_sm is not None or event_passes is not None:
            wbrw_set_tuning(self.ctx, b if blocks_per_sm is None else blocks_per_sm,
                            p if event_passes is None else event_passes)
            b, p = wbrw_get_tuning(self.ctx)
        return b, p

    def graph(self, enable=True):
        """Replay resampling periods from CUDA graphs (needs a created stream)."""
        wbrw_graph(self.ctx, enable)

    def one_launch_periods(self, enable=True):
        """Run regenerating periods as one launch where the kernels allow
        (the default), or launch per round (the same results)."""
        wbrw_one_launch_periods(self.ctx, enable)

    def density(self):
        return wbrw_density(self.ctx, self.nx, self.nk)

    def counters(self):
        return wbrw_counters(self.ctx)

    def checkpoint(self, grid_out=None):
        """Copy the histogram into grid_out (host or device int32 array-like
        with a data pointer; a new host array if None); returns (grid, step, epoch)."""
        if grid_out is None:
            grid_out = np.empty(((self.ninst,) if self.ninst > 1 else ()) + (self.nx, self.nk),
                                np.int32)
        ptr = grid_out.ctypes.data if isinstance(grid_out, np.ndarray) else grid_out.data_ptr()
        step, epoch = wbrw_checkpoint(self.ctx, ptr)
        return grid_out, step, epoch

    def restore(self, grid, step, epoch):
        if isinstance(grid, np.ndarray):
            grid = np.ascontiguousarray(grid, np.int32)
            self._restore_keep = grid
            ptr = grid.ctypes.data
        else:
            ptr = grid.data_ptr()
            self.stream.wait_stream(self.torch.cuda.current_stream())
        wbrw_restore(self.ctx, ptr, step, epoch)

    def particles(self, with_pids=True):
        """(x, k, s, w, pid) of the current particles as host numpy arrays."""
        torch = self.torch
        n = wbrw_particles(self.ctx)
        pid = None
        if with_pids:
            pid_t = torch.empty(max(n, 1), dtype=torch.int64, device=self.x.device)
            wbrw_particles(self.ctx, pid_t.data_ptr())
            pid = pid_t[:n].cpu().numpy().view(np.uint64)
        x = self.x[:n].cpu().numpy()
        k = self.k[:n].cpu().numpy()
        s = self.s[:n].cpu().numpy()
        w = self.w[:n].cpu().numpy() if self.w is not None else s.astype(x.dtype)
        return x, k, s, w, pid

    def transmission_gradients(self):
        """(dT/dH, dT/dw) per instance after a resampling (tangent mode)."""
        g = wbrw_transmission_gradients(self.ctx, self.ninst)
        return g if self.ninst > 1 else g[0]

    def tangents(self):
        """(tau_H, tau_w) of the materialised particles (tangent mode)."""
        n = wbrw_particles(self.ctx)
        c = self.capacity
        return self.tan[:n].cpu().numpy(), self.tan[c:c + n].cpu().numpy()

    def grid_counts(self):
        self.stream.synchronize()
        if self.ninst > 1:
            return self.grid.view(self.ninst, self.nx, self.nk).cpu().numpy()
        return self.grid.view(self.nx, self.nk).cpu().numpy()

    def event_log(self):
        c = self.counters()
        n = min(c["log_len"], self.bufs.event_log_capacity)
        if self.log is None or n == 0:
            return np.zeros(0, EVENT_DTYPE)
        raw = self.log[: n * EVENT_DTYPE.itemsize].cpu().numpy()
        return raw.view(EVENT_DTYPE).copy()

    def close(self):
        if getattr(self, "ctx", None):
            wbrw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Simulation):
    """Many independent problems in the same launches (any strategy).

    ``wl`` gives the shared configuration (precision, dt, grid, seed, ...);
    ``instances`` is a list of dicts with keys H, w, xc, x0, sigma_x, k0,
    n_init, n_alpha and optionally gamma0 (default: the majorant C/2).
    """

    def __init__(self, wl: dict, instances, capacity: int, *, event_log: int = 0, stream=None):
        self.ninst = len(instances)
        self._buffers(wl, capacity, event_log, stream)
        self.instances = [dict(v) for v in instances]
        recs = [Instance(Potential(POT_GAUSSIAN, v["H"], v["w"], v.get("xc", 0.0)),
                         v["x0"], v["sigma_x"], v["k0"], int(v["n_init"]), int(v["n_alpha"]),
                         v.get("gamma0", 0.0)) for v in instances]
        self.ctx = wbrw_batch_init(self.cfg, recs, self.bufs, self.stream.cuda_stream)

    def density(self, inst=0):
        return wbrw_instance_density(self.ctx, inst, self.nx, self.nk)

    def transmissions(self):
        return wbrw_transmissions(self.ctx, self.ninst)

    def particles(self, with_pids=True):
        """(x, k, s, w, pid, inst) of the current particles as host arrays."""
        x, k, s, w, pid = super().particles(with_pids)
        t = self.torch.empty(max(len(x), 1), dtype=self.torch.int32, device=self.x.device)
        wbrw_particle_instances(self.ctx, t.data_ptr())
        return x, k, s, w, pid, t[: len(x)].cpu().numpy().view(np.uint32)


class Simulation4(Simulation):
    """The 4D Helium-like system: two electrons (x1, x2, k1, k2) around a
    nucleus, soft-Coulomb one-body terms of charge Z and an interaction of
    strength ee, softening a (workloads.HE_4D_*)."""

    def __init__(self, wl: dict, capacity: int, *, event_log: int = 0, stream=None):
        wl = dict(wl, dim=4)
        self._buffers(wl, capacity, event_log, stream)
        self.pot = Potential(POT_SOFT_COULOMB_2E, wl["Z"], wl["a"], wl["xc"], wl["lam"])
        self.ctx = wbrw_init4d(self.cfg, self.pot, self.bufs, int(wl["n_alpha"]),
                               tuple(wl["x0"]), wl["sigma_x"], tuple(wl["k0"]),
                               self.stream.cuda_stream)

    def particles(self, with_pids=True):
        """(x1, x2, k1, k2, s, pid) of the current particles as host arrays."""
        torch = self.torch
        n = wbrw_particles(self.ctx)
        pid = None
        if with_pids:
            pid_t = torch.empty(max(n, 1), dtype=torch.int64, device=self.x.device)
            wbrw_particles(self.ctx, pid_t.data_ptr())
            pid = pid_t[:n].cpu().numpy().view(np.uint64)
        c = self.capacity
        x1, x2 = self.x[:n].cpu().numpy(), self.x[c:c + n].cpu().numpy()
        k1, k2 = self.k[:n].cpu().numpy(), self.k[c:c + n].cpu().numpy()
        s = self.s[:n].cpu().numpy()
        return x1, x2, k1, k2, s, pid

    def grid_counts(self):
        self.stream.synchronize()
        return self.grid.view(self.nx, self.nx, self.nk, self.nk).cpu().numpy()

    def checkpoint(self, grid_out=None):
        if grid_out is None:
            grid_out = np.empty((self.nx, self.nx, self.nk, self.nk), np.int32)
        return super().checkpoint(grid_out)
