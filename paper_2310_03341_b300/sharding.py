"""Sharding of independent BdG blocks (kz blocks, SCF replicas) over the ranks of a
torch.distributed group: one process per GPU, no collective inside a solve.

partition_blocks  assigns blocks to ranks greedily by cost n^3, largest first (each block goes to
                  the rank with the least work so far), so that every rank gets a contiguous
                  share of the total work;
gather_spectra    all-gathers the eigenvalues each rank computed, so every rank holds the whole
                  spectrum in the original block order (the one exchange step of the batched
                  path);
max_over_ranks    the timing reduction of the benchmark (the slowest rank sets the time).
"""
from __future__ import annotations

import numpy as np


def partition_blocks(sizes, world: int):
    """List of block indices per rank (greedy by n^3, largest first)."""
    load = [0.0] * world
    owned = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(i)
        load[r] += float(sizes[i]) ** 3
    return [sorted(o) for o in owned]


def gather_spectra(local: dict, sizes, world: int, group=None):
    """local: {block index: eigenvalues (float64 array)} of this rank -> list of all blocks'
    eigenvalues in block order, on every rank (one all_gather of a padded buffer)."""
    import torch
    import torch.distributed as dist
    total = int(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    buf = torch.zeros(total + 1, dtype=torch.float64)
    for i, ev in local.items():
        buf[offs[i]:offs[i + 1]] = torch.as_tensor(np.asarray(ev, dtype=np.float64))
    mine = torch.zeros(total + 1, dtype=torch.float64)
    mine[:] = buf
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    owner = np.full(len(sizes), -1)
    flags = torch.zeros(len(sizes), dtype=torch.int64)
    for i in local:
        flags[i] = 1
    allf = [torch.zeros_like(flags) for _ in range(world)]
    dist.all_gather(allf, flags, group=group)
    for r in range(world):
        owner[allf[r].numpy() == 1] = r
    if np.any(owner < 0):
        raise RuntimeError("gather_spectra: a block was solved by no rank")
    return [parts[owner[i]][offs[i]:offs[i + 1]].numpy().copy() for i in range(len(sizes))]


def max_over_ranks(value: float, device=None, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
