"""The allocation-free observables entry point.

Some callers cannot call cudaMalloc: code running inside a device memory pool
owned by someone else, or a process that must not grow its device footprint
after start-up.  wbrw_observables_static serves them: its only scratch is a
static device array inside the library, so the caller passes just the
histogram and the output buffers.  This test calls it through the C ABI twice
in a row, on two different histograms, and checks each result against the
observables that wbrw_density returns for the same state.  The density is a
ratio of integers and the transmission an exact integer sum divided once, so
the comparison is exact, as in the other observables tests.
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


def test_static_observables_match_density_twice(torch):
    from paper_1709_02121_gb300 import Simulation, wbrw
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=4100, nx=100, nk=64,
                          xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2, resample_every=5)
    sim = Simulation(wl, capacity=200_000)
    nx, nk = wl["nx"], wl["nk"]
    dens_d = torch.zeros(nx * nk, dtype=torch.float64, device="cuda")
    marg_d = torch.zeros(nx, dtype=torch.float64, device="cuda")
    T_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.run(5)                      # a new histogram for each call
        dens, marg, T, _ = sim.density()
        st = wbrw.wbrw_observables_static(
            sim.grid.data_ptr(), nx, nk, wl["xmin"], wl["xmax"], wl["kmin"], wl["kmax"],
            wl["n_alpha"], dens_d.data_ptr(), marg_d.data_ptr(), T_d.data_ptr(),
            sim.stream.cuda_stream)
        assert st == wbrw.OK
        torch.cuda.synchronize()
        assert np.array_equal(dens_d.cpu().numpy().reshape(nx, nk), dens), call
        assert np.array_equal(marg_d.cpu().numpy(), marg), call
        assert T_d.item() == T, call
        assert np.abs(dens).sum() > 0


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
