"""Sharding of independent BdG blocks (kz blocks, SCF replicas) over the ranks of a
torch.distributed group: one process per GPU, no collective inside a solve.

partition_blocks  assigns blocks to ranks greedily by cost n^3, largest first (each block goes to
                  the rank with the least work so far), so that every rank gets a contiguous
                  share of the total work;
gather_spectra    all-gathers the eigenvalues each rank computed, so every rank holds the whole
                  spectrum in the original block order (the one exchange step of the batched
                  path);
solve_sharded     the batched path over ranks: partition, build and solve only the owned blocks
                  (one batched call per rank), then gather the eigenvalues; eigenvectors stay on
                  the rank that computed them;
reduce_densities  sums the partial densities (n, nu) that each rank accumulated over its own blocks
                  into the full densities on every rank (one all_reduce);
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


def gather_spectra(local: dict, sizes, world: int, group=None, device=None):
    """local: {block index: eigenvalues (float64 array)} of this rank -> list of all blocks'
    eigenvalues in block order, on every rank (one all_gather of a padded buffer, one of the
    ownership flags).  device: where the exchanged buffers live (None: host memory, as gloo
    wants; the rank's CUDA device under NCCL).  A block that no rank or two ranks report is an
    error."""
    import torch
    import torch.distributed as dist
    total = int(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    mine = torch.zeros(total + 1, dtype=torch.float64)
    flags = torch.zeros(len(sizes), dtype=torch.int64)
    for i, ev in local.items():
        mine[offs[i]:offs[i + 1]] = torch.as_tensor(np.asarray(ev, dtype=np.float64)).reshape(-1)
        flags[i] = 1
    if device is not None:
        mine, flags = mine.to(device), flags.to(device)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    allf = [torch.zeros_like(flags) for _ in range(world)]
    dist.all_gather(allf, flags, group=group)
    allf = np.stack([f.cpu().numpy() for f in allf])
    if np.any(allf.sum(axis=0) != 1):
        raise RuntimeError("gather_spectra: every block must be solved by exactly one rank")
    owner = allf.argmax(axis=0)
    return [parts[owner[i]][offs[i]:offs[i + 1]].cpu().numpy().copy() for i in range(len(sizes))]


def solve_sharded(sizes, make_block, solve_batch, rank: int, world: int, group=None,
                  device=None):
    """The batched path over `world` ranks, called on every rank.

    sizes        dimension of every block (the same list on every rank);
    make_block   i -> block i as a matrix on this rank's device (called only for owned blocks,
                 so no rank holds the others' matrices);
    solve_batch  list of matrices -> list of (w, Z) (one batched eigensolve, e.g.
                 Context.heev_batched);
    returns (spectra, local): every block's eigenvalues in block order on every rank, and
    {i: (w, Z)} for the blocks this rank solved.  A rank that owns no block still joins the
    exchange.
    """
    mine = partition_blocks(sizes, world)[rank]
    out = solve_batch([make_block(i) for i in mine]) if mine else []
    if len(out) != len(mine):
        raise RuntimeError("solve_sharded: the batched solve returned the wrong number of blocks")
    local = dict(zip(mine, out))
    ev = {i: np.asarray(w.cpu() if hasattr(w, "cpu") else w, dtype=np.float64)
          for i, (w, _) in local.items()}
    return gather_spectra(ev, sizes, world, group, device), local


def reduce_densities(n, nu, group=None):
    """n (real) and nu (complex) partial densities of this rank's blocks -> their sums over all
    ranks, in place and returned (one all_reduce of [n, Re nu, Im nu] packed in one buffer).  The
    tensors may live on the host (gloo) or on the rank's device (NCCL); a rank that owns no block
    passes zeros."""
    import torch
    import torch.distributed as dist
    V = n.numel()
    if nu.numel() != V:
        raise ValueError("reduce_densities: n and nu must have one entry per site")
    buf = torch.empty(3 * V, dtype=torch.float64, device=n.device)
    buf[:V] = n.reshape(-1)
    buf[V:] = torch.view_as_real(nu.reshape(-1)).transpose(0, 1).reshape(-1)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    n.copy_(buf[:V].reshape(n.shape))
    nu.copy_(torch.complex(buf[V:2 * V], buf[2 * V:]).reshape(nu.shape))
    return n, nu


def max_over_ranks(value: float, device=None, group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
