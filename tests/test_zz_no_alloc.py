"""The allocation-free observables entry point.

Some callers cannot call cudaMalloc: code running inside a device memory pool
owned by someone else, or a process that must not grow its device footprint
after start-up.  wbrw_observables_static serves them: its only scratch is a
static device array inside the library, so the caller passes just the
histogram and the output buffers.  These tests call it through the C ABI:
twice in a row on two different histograms against the observables that
wbrw_density returns for the same state, without the optional density, at the
largest nx it accepts against the oracle, with the device's free memory
unchanged across a call, and with buffers that are not device memory.  The
density is a ratio of integers and the transmission an exact integer sum
divided once, so every comparison is exact, as in the other observables
tests.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def _static(wbrw, grid, nx, nk, lims, n_alpha, dens, marg, T, stream=0):
    return wbrw.wbrw_observables_static(
        grid.data_ptr(), nx, nk, lims[0], lims[1], lims[2], lims[3], n_alpha,
        dens.data_ptr() if dens is not None else 0, marg.data_ptr(), T.data_ptr(), stream)


def test_static_observables_match_density_twice(torch):
    from paper_1709_02121_gb300 import Simulation, wbrw
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=4100, nx=100, nk=64,
                          xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2, resample_every=5)
    sim = Simulation(wl, capacity=200_000)
    nx, nk = wl["nx"], wl["nk"]
    lims = (wl["xmin"], wl["xmax"], wl["kmin"], wl["kmax"])
    dens_d = torch.zeros(nx * nk, dtype=torch.float64, device="cuda")
    marg_d = torch.zeros(nx, dtype=torch.float64, device="cuda")
    T_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.run(5)                      # a new histogram for each call
        dens, marg, T, _ = sim.density()
        st = _static(wbrw, sim.grid, nx, nk, lims, wl["n_alpha"], dens_d, marg_d, T_d,
                     sim.stream.cuda_stream)
        assert st == wbrw.OK
        torch.cuda.synchronize()
        assert np.array_equal(dens_d.cpu().numpy().reshape(nx, nk), dens), call
        assert np.array_equal(marg_d.cpu().numpy(), marg), call
        assert T_d.item() == T, call
        assert np.abs(dens).sum() > 0
    # the density is optional: marginal and transmission alone
    marg_d.zero_()
    T_d.zero_()
    st = _static(wbrw, sim.grid, nx, nk, lims, wl["n_alpha"], None, marg_d, T_d,
                 sim.stream.cuda_stream)
    assert st == wbrw.OK
    torch.cuda.synchronize()
    assert np.array_equal(marg_d.cpu().numpy(), marg)
    assert T_d.item() == T
    sim.close()


def test_static_observables_at_the_largest_nx_match_the_oracle(torch):
    """nx = WBRW_STATIC_MAX_NX uses the last entry of the static array.  x = 0
    falls on a cell edge of [-40, 24), so the transmission is the sum of the
    columns right of it."""
    import oracle
    from paper_1709_02121_gb300 import wbrw
    nx, nk, n_alpha = 65536, 1, 123457
    lims = (-40.0, 24.0, -3.0, 5.0)
    rng = np.random.default_rng(7)
    g = rng.integers(-50, 51, size=nx * nk).astype(np.int32)
    o = oracle.Oracle(nx=nx, nk=nk, xmin=lims[0], xmax=lims[1], kmin=lims[2], kmax=lims[3],
                      n_alpha=n_alpha)
    odens, omarg, oT = o.observables(g.reshape(nx, nk))
    grid = torch.from_numpy(g).cuda()
    dens = torch.zeros(nx * nk, dtype=torch.float64, device="cuda")
    marg = torch.zeros(nx, dtype=torch.float64, device="cuda")
    T = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert _static(wbrw, grid, nx, nk, lims, n_alpha, dens, marg, T) == wbrw.OK
    torch.cuda.synchronize()
    assert np.array_equal(dens.cpu().numpy().reshape(nx, nk), odens)
    assert np.array_equal(marg.cpu().numpy(), omarg)
    assert T.item() == oT
    # the last column is the last entry of the static scratch
    assert marg[-1].item() == g[-1] / (n_alpha * (lims[1] - lims[0]) / nx)
    assert oT == g[nx * 40 // 64:].astype(np.int64).sum() / n_alpha


def test_static_observables_allocate_nothing(torch):
    """After one call has loaded the kernels, a further call leaves the
    device's free memory exactly as it was."""
    from paper_1709_02121_gb300 import wbrw
    nx, nk = 600, 256
    lims = (-60.0, 60.0, -6.4, 6.4)
    g = torch.randint(-9, 10, (nx * nk,), dtype=torch.int32, device="cuda")
    dens = torch.empty(nx * nk, dtype=torch.float64, device="cuda")
    marg = torch.empty(nx, dtype=torch.float64, device="cuda")
    T = torch.empty(1, dtype=torch.float64, device="cuda")
    assert _static(wbrw, g, nx, nk, lims, 1000, dens, marg, T) == wbrw.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _static(wbrw, g, nx, nk, lims, 1000, dens, marg, T) == wbrw.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_observables_reject_oversized_and_bad_arguments(torch):
    from paper_1709_02121_gb300 import wbrw
    g = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    big = wbrw.wbrw_observables_static(g.data_ptr(), 65537, 1, -1.0, 1.0, -1.0, 1.0, 10,
                                       0, out.data_ptr(), out.data_ptr(), 0)
    assert big == wbrw.ERR_CAPACITY
    bad = wbrw.wbrw_observables_static(g.data_ptr(), 0, 1, -1.0, 1.0, -1.0, 1.0, 10,
                                       0, out.data_ptr(), out.data_ptr(), 0)
    assert bad == wbrw.ERR_ARG
    # buffers in host memory (pageable and pinned) are refused before any
    # launch, so no kernel ever touches them
    gh = np.zeros(8, np.int32)
    st = wbrw.wbrw_observables_static(gh.ctypes.data, 8, 1, -1.0, 1.0, -1.0, 1.0, 10,
                                      0, out.data_ptr(), out.data_ptr(), 0)
    assert st == wbrw.ERR_ARG
    pinned = torch.zeros(8, dtype=torch.float64).pin_memory()
    st = wbrw.wbrw_observables_static(g.data_ptr(), 8, 1, -1.0, 1.0, -1.0, 1.0, 10,
                                      0, pinned.data_ptr(), out.data_ptr(), 0)
    assert st == wbrw.ERR_ARG
    st = wbrw.wbrw_observables_static(g.data_ptr(), 8, 1, -1.0, 1.0, -1.0, 1.0, 10,
                                      pinned.data_ptr(), out.data_ptr(), out.data_ptr(), 0)
    assert st == wbrw.ERR_ARG
    # the refusals leave no error behind: a valid call still succeeds
    st = wbrw.wbrw_observables_static(g.data_ptr(), 8, 1, -1.0, 1.0, -1.0, 1.0, 10,
                                      0, out.data_ptr(), out.data_ptr(), 0)
    assert st == wbrw.OK
    torch.cuda.synchronize()
