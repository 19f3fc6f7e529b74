"""Splitting a batch of walls across ranks (one process per GPU).

Walls are independent, so a batch shards with no exchange in the data path: each rank advances its own
walls, and only the host-side results (fields, fluxes, samples, timings) are gathered. The partition
balances the node counts (the work of a wall is proportional to its nodes).
"""
from __future__ import annotations

import numpy as np


def partition_walls(n_nodes, world: int) -> list[np.ndarray]:
    """Wall indices of each rank: longest-processing-time-first by node count, each rank's list sorted."""
    n_nodes = np.asarray(n_nodes, np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = np.zeros(world, np.int64)
    parts: list[list[int]] = [[] for _ in range(world)]
    for w in np.argsort(-n_nodes, kind="stable"):
        r = int(np.argmin(load))
        parts[r].append(int(w))
        load[r] += n_nodes[w]
    return [np.array(sorted(p), np.int64) for p in parts]


def shard(wl, rank: int, world: int):
    """The rank's walls of workload ``wl`` and their indices in the whole batch."""
    idx = partition_walls(wl.n_nodes, world)[rank]
    return wl.subset(idx), idx


def gather_walls(pg, idx: np.ndarray, per_wall: np.ndarray, n_walls: int, rank: int) -> np.ndarray | None:
    """Rank 0 receives every rank's per-wall rows ([len(idx), ...]) placed at their batch positions."""
    import torch

    rows = torch.from_numpy(np.ascontiguousarray(per_wall, np.float64))
    ids = torch.from_numpy(np.ascontiguousarray(idx, np.int64))
    world = pg.get_world_size()
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    pg.all_gather(sizes, torch.tensor([len(idx)], dtype=torch.int64))
    m = int(max(s.item() for s in sizes))
    pad_rows = torch.zeros((m,) + tuple(rows.shape[1:]), dtype=torch.float64)
    pad_rows[: len(idx)] = rows
    pad_ids = torch.full((m,), -1, dtype=torch.int64)
    pad_ids[: len(idx)] = ids
    all_rows = [torch.zeros_like(pad_rows) for _ in range(world)]
    all_ids = [torch.zeros_like(pad_ids) for _ in range(world)]
    pg.all_gather(all_rows, pad_rows)
    pg.all_gather(all_ids, pad_ids)
    if rank != 0:
        return None
    out = np.zeros((n_walls,) + tuple(rows.shape[1:]))
    for r in range(world):
        k = int(sizes[r].item())
        out[all_ids[r][:k].numpy()] = all_rows[r][:k].numpy()
    return out


def node_slices(wl, idx: np.ndarray, values: np.ndarray) -> list[np.ndarray]:
    """Per-wall slices of a concatenated node array of the sub-batch ``wl`` (walls ``idx``)."""
    off = np.concatenate([[0], np.cumsum(wl.n_nodes)])
    return [values[off[i]: off[i + 1]] for i in range(len(idx))]
