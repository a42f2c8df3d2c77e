"""The lean FP32 kernels give the general kernels' results bit for bit.

An FP32 2D run (plain or batched, with or without tangents) with the static
potential and no event log runs kernels compiled without the time-dependent
components and the log writes (without tangents: built for four blocks per
SM), whose event kernel finishes deferred segments itself.  Attaching an event log (which changes no result) selects the
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


@pytest.mark.parametrize("batch", [False, True])
def test_lean_tangent_kernels_equal_the_general_ones(torch, batch):
    """Tangent mode: the lean kernels (static potential, no event log) finish
    deferred segments inside the event kernel too; the histograms, the
    gradients, the counters and the particles with their tangent weights are
    those of the general tangent kernels."""
    from paper_1709_02121_gb300 import Batch, Simulation
    wl = workloads.scaled(workloads.COLLISION_2D, precision="fp32", n_alpha=20_000, gamma0=2.0,
                          nx=100, nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2,
                          resample_every=5, tangent=True, tquantum=0.5)
    if batch:
        insts = [dict(H=h, w=v, xc=0.0, x0=wl["x0"], sigma_x=wl["sigma_x"], k0=wl["k0"],
                      n_init=8000, n_alpha=8000) for h, v in ((1.0, 1.0), (0.6, 1.4), (1.5, 0.8))]

        def make(**kw):
            return Batch(wl, insts, 3_000_000, stream=torch.cuda.Stream(), **kw)
    else:
        def make(**kw):
            return Simulation(wl, 2_000_000, stream=torch.cuda.Stream(), **kw)
    lean, gen = make(), make(event_log=1 << 16)
    lean.graph(True)
    gen.graph(True)
    for period in range(4):
        lean.run(5)
        gen.run(5)
        assert np.array_equal(lean.grid_counts(), gen.grid_counts()), period
        assert np.array_equal(lean.transmission_gradients(), gen.transmission_gradients()), period
    a, b = lean.counters(), gen.counters()
    for k in KEYS[:12]:
        assert a[k] == b[k], k
    assert b["log_len"] > 0
    lean.step(3)
    gen.step(3)
    pa, pb = lean.particles()[4], gen.particles()[4]
    ia, ib = np.argsort(pa, kind="stable"), np.argsort(pb, kind="stable")
    assert np.array_equal(pa[ia], pb[ib])
    for u, v in zip(lean.tangents(), gen.tangents()):
        assert np.array_equal(u[ia], v[ib])
    lean.close()
    gen.close()


@pytest.mark.parametrize("kind,strategy", [("plain", "sp1"), ("plain", "wp"), ("batch", "sp1"),
                                           ("batch", "wp"), ("tangent", "sp1")])
def test_one_launch_periods_equal_the_launch_per_round_schedule(torch, kind, strategy):
    """The lean kernels run a regenerating sp1 or wp period (into the signed
    histogram or the weight sums) as one launch; the launch-per-round
    schedule of the same kernels gives the same results."""
    from paper_1709_02121_gb300 import Batch, Simulation
    wl = workloads.scaled(workloads.GAUSS_2D_FP64_2E5, precision="fp32", n_alpha=20_000, nx=100,
                          nk=64, xmin=-25.0, xmax=25.0, kmin=-3.2, kmax=3.2, resample_every=5,
                          strategy=strategy, tangent=kind == "tangent", tquantum=0.5)
    if kind == "plain":
        def make():
            return Simulation(wl, 2_000_000, stream=torch.cuda.Stream())
    else:
        insts = [dict(H=h, w=v, xc=0.0, x0=wl["x0"], sigma_x=wl["sigma_x"], k0=wl["k0"],
                      n_init=8000, n_alpha=8000) for h, v in ((1.0, 1.0), (0.6, 1.4), (1.5, 0.8))]

        def make():
            return Batch(wl, insts, 3_000_000, stream=torch.cuda.Stream())
    a, b = make(), make()
    b.one_launch_periods(False)
    for s_ in (a, b):
        s_.graph(True)
    for period in range(4):
        a.run(5)
        b.run(5)
        assert np.array_equal(a.grid_counts(), b.grid_counts()), period
        if kind == "tangent":
            assert np.array_equal(a.transmission_gradients(), b.transmission_gradients()), period
    ca, cb = a.counters(), b.counters()
    for k in KEYS[:12] if kind != "plain" else KEYS:
        assert ca[k] == cb[k], k
    a.close()
    b.close()
