"""The lean FP32 kernels give the general kernels' results bit for bit.

An FP32 2D run (plain or batched) with the static potential and no event log
runs kernels compiled without the time-dependent components and the log
writes, built for four blocks per SM, whose event kernel finishes deferred
segments itself.  Attaching an event log (which changes no result) selects the
general kernels for the same run, so the two can be compared on the same
streams: histograms after every period, the counters, and the particles after
plain steps.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

KEYS = ("events", "kill_plus", "kill_minus", "out_plus", "out_minus", "particle_steps",
        "particle_steps_first", "live", "step", "epoch", "candidates", "first_pairs",
        "boot_nplus", "boot_nminus", "boot_nrplus", "boot_nrminus", "boot_wplus", "boot_wminus")


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_02121_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("strategy", ["sp1", "sp2", "wp"])
def test_lean_kernels_equal_the_general_ones(torch, strategy):
    from paper_1709_02121_gb300 import Simulation
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, precision="fp32", strategy=strategy,
                          n_alpha=20_000, nx=100, nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2,
                          kmax=3.2, resample_every=5)
    lean = Simulation(wl, 2_000_000, stream=torch.cuda.Stream())
    gen = Simulation(wl, 2_000_000, event_log=1 << 16, stream=torch.cuda.Stream())
    lean.graph(True)
    gen.graph(True)
    for period in range(5):
        lean.run(5)
        gen.run(5)
        assert np.array_equal(lean.grid_counts(), gen.grid_counts()), period
    a, b = lean.counters(), gen.counters()
    for k in KEYS:
        assert a[k] == b[k], k
    assert b["log_len"] > 0          # the general kernels did write the log
    lean.step(3)
    gen.step(3)
    xa, ka, sa, wa, pa = lean.particles()
    xb, kb, sb, wb, pb = gen.particles()
    ia, ib = np.argsort(pa, kind="stable"), np.argsort(pb, kind="stable")
    assert np.array_equal(pa[ia], pb[ib])
    for u, v in ((xa, xb), (ka, kb), (sa, sb)):
        assert np.array_equal(u[ia], v[ib])
    lean.close()
    gen.close()


def test_lean_batch_equals_the_general_batch(torch):
    from paper_1709_02121_gb300 import Batch
    wl = workloads.scaled(workloads.BATCH_2D_FP32_256, nx=100, nk=64, xmin=-25.0, xmax=25.0,
                          kmin=-3.2, kmax=3.2, resample_every=5)
    insts = workloads.batch_instances(dict(wl, instances=5), 0.004)
    lean = Batch(wl, insts, 3_000_000, stream=torch.cuda.Stream())
    gen = Batch(wl, insts, 3_000_000, event_log=1 << 16, stream=torch.cuda.Stream())
    lean.graph(True)
    gen.graph(True)
    for period in range(4):
        lean.run(5)
        gen.run(5)
        assert np.array_equal(lean.grid_counts(), gen.grid_counts()), period
        assert np.array_equal(lean.transmissions(), gen.transmissions()), period
    a, b = lean.counters(), gen.counters()
    for k in KEYS[:12]:
        assert a[k] == b[k], k
    lean.close()
    gen.close()
