"""Non-finite particle state is detected, not binned silently.

A particle whose position or wavevector is NaN or infinite fails every
comparison of the cell test, so binning would drop it as if it had left the
grid.  The binning sink latches WBRW_ERR_NUMERIC in the device error word
instead; the next synchronising call reports it and the context refuses
further work.  The bad values are written by the host into the caller's
particle arrays between two calls, so nothing on the device faults or traps:
the kernels only read the values and record the error.
"""
import math

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


def _sim(precision):
    from paper_1709_02121_gb300 import Simulation
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, precision=precision, n_alpha=4100,
                          nx=100, nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2)
    return Simulation(wl, capacity=200_000)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("where,value", [("x", math.nan), ("k", math.inf),
                                         ("x", -math.inf)])
def test_non_finite_state_is_reported(torch, precision, where, value):
    from paper_1709_02121_gb300 import WbrwError, wbrw
    sim = _sim(precision)
    sim.step(2)
    n = sim.counters()["live"]
    assert wbrw.wbrw_sync_status(sim.ctx) == wbrw.OK
    arr = sim.x if where == "x" else sim.k
    arr[n // 2] = value                       # the host writes the bad value
    sim.stream.wait_stream(torch.cuda.current_stream())
    sim.step(1)
    sim.annihilate()
    assert wbrw.wbrw_sync_status(sim.ctx) == wbrw.ERR_NUMERIC
    assert "non-finite" in wbrw.wbrw_last_error(sim.ctx)
    with pytest.raises(WbrwError) as ei:
        sim.step(1)
    assert ei.value.status == wbrw.ERR_STATE
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_finite_particles_outside_the_grid_are_no_error(torch, precision):
    """A finite particle far outside the grid is dropped and tallied, as
    before; only non-finite values raise the error."""
    from paper_1709_02121_gb300 import wbrw
    sim = _sim(precision)
    sim.step(2)
    n = sim.counters()["live"]
    sim.x[n // 2] = 1e30
    sim.k[n // 3] = -1e30
    sim.stream.wait_stream(torch.cuda.current_stream())
    out0 = sim.counters()["out_plus"] + sim.counters()["out_minus"]
    sim.step(1)
    sim.annihilate()
    assert wbrw.wbrw_sync_status(sim.ctx) == wbrw.OK
    c = sim.counters()
    assert c["out_plus"] + c["out_minus"] >= out0 + 2
    sim.close()
