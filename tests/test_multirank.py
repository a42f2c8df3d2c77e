"""Multi-rank paths on CPU ranks (gloo, world size 2).

The method shards by particles between resamplings and merges the
processors' histograms by an integer sum (Sec. 4).  Because every random draw
is keyed by particle id, ranks that each step a share of the particles and
all-reduce their int32 counts must reproduce the single-process histogram
exactly.  The benchmark's replica reduction (max time, summed work) is checked
on the same backend."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _wl():
    return workloads.scaled(workloads.GAUSS_2D_FP64_2E5, n_alpha=3000, nx=80, nk=64,
                            xmin=-40.0, xmax=0.0, kmin=-3.2, kmax=3.2)


def _oracle_share(wl, rank, world):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import make_oracle
    full = make_oracle(wl)
    full.init_gauss(wl["n_alpha"], wl["x0"], wl["sigma_x"], wl["k0"])
    x, k, w, pid = full.particles()
    mine = (pid % np.uint64(world)) == np.uint64(rank)
    o = make_oracle(wl)
    o.set_particles(x[mine], k[mine], w[mine], pid[mine], step=0)
    o.step(6)
    counts, _ = o.histogram()
    return counts, o.ledger()


def _rank_main(rank, world, port, wl, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    counts, led = _oracle_share(wl, rank, world)
    c = torch.from_numpy(counts.astype(np.int64)).reshape(-1)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    ev = torch.tensor([led["events"], led["particle_steps"]], dtype=torch.int64)
    dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    import bench
    t, ps, e2e = bench.reduce_over_ranks(world, 10.0 + rank, 100 * (rank + 1), 1.5, "cpu")
    if rank == 0:
        np.save(out + ".counts.npy", c.numpy())
        np.save(out + ".ledger.npy", ev.numpy())
        np.save(out + ".bench.npy", np.array([t, ps, e2e]))
    dist.destroy_process_group()


def test_sharded_histograms_merge_to_the_single_process_one(tmp_path, oracle_mod):
    wl = _wl()
    out = str(tmp_path / "merge")
    mp.start_processes(_rank_main, args=(2, _free_port(), wl, out), nprocs=2, join=True,
                       start_method="spawn")
    merged = np.load(out + ".counts.npy").reshape(wl["nx"], wl["nk"])
    single, led = _oracle_share(wl, 0, 1)
    assert np.array_equal(merged, single.astype(np.int64))
    ev = np.load(out + ".ledger.npy")
    assert ev[0] == led["events"] and ev[1] == led["particle_steps"]
    assert np.abs(single).sum() > 1000
    t, ps, e2e = np.load(out + ".bench.npy")
    assert t == 11.0 and ps == 300 and e2e == 3.0
