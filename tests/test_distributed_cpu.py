"""The multi-rank path on CPU ranks (gloo, world size 2): a batch split by the partitioner, each rank
advancing its own walls, results gathered on rank 0 -- equal to the single-process run. The ranks use
the FP64 oracle as their engine (there is no GPU here); the split and the gather are the same code a GPU
rank uses. Also the benchmark's cross-rank timing reductions (max of times, sum of units)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1703_10119_gb300 import shard
    from paper_1703_10119_gb300 import workloads as wk

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = wk.wall_batch(seed=21, n_walls=12, n_steps=60, n_min=5, n_max=40)
    sub, idx = shard.shard(wl, rank, world)
    o = oracle.Oracle(sub, n_threads=1)
    r = o.run(60, 20)
    flux = shard.gather_walls(dist, idx, r["flux"], wl.n_walls, rank)
    samples = shard.gather_walls(dist, idx, np.moveaxis(r["samples"], 1, 0), wl.n_walls, rank)
    Tl = shard.node_slices(sub, idx, o.T_cur)
    width = int(wl.n_nodes.max())
    T = np.full((len(idx), width), np.nan)
    for i, t in enumerate(Tl):
        T[i, : len(t)] = t
    Tall = shard.gather_walls(dist, idx, T, wl.n_walls, rank)
    # the benchmark's reductions: max of the ranks' times, sum of their units
    tmax = bench.reduce_max(dist, float(1 + rank))
    usum = bench.reduce_sum(dist, float(10 * (rank + 1)))
    if rank == 0:
        np.savez(os.path.join(out_dir, "rank0.npz"), flux=flux, samples=samples, T=Tall, tmax=tmax, usum=usum)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_balances_nodes():
    from paper_1703_10119_gb300 import shard

    rng = np.random.default_rng(0)
    n = rng.integers(50, 401, 4096)
    for world in (1, 2, 3, 8):
        parts = shard.partition_walls(n, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(len(n)))
        loads = np.array([n[p].sum() for p in parts])
        assert loads.max() - loads.min() <= n.max()


def test_two_rank_split_equals_single_process(tmp_path, oracle_mod):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "rank0.npz")
    from paper_1703_10119_gb300 import workloads as wk

    wl = wk.wall_batch(seed=21, n_walls=12, n_steps=60, n_min=5, n_max=40)
    o = oracle_mod.Oracle(wl, n_threads=1)
    r = o.run(60, 20)
    assert np.array_equal(got["flux"], r["flux"])
    assert np.array_equal(got["samples"], np.moveaxis(r["samples"], 1, 0))
    off = np.concatenate([[0], np.cumsum(wl.n_nodes)])
    for w in range(wl.n_walls):
        n = wl.n_nodes[w]
        assert np.array_equal(got["T"][w, :n], o.T_cur[off[w]: off[w + 1]])
    assert float(got["tmax"]) == 2.0 and float(got["usum"]) == 30.0
