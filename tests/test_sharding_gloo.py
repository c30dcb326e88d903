"""Multi-rank host logic on CPU (gloo, world size 2): block partition,
eigenvalue all-gather of the batched path, and the benchmark's max-over-ranks
timing.  The per-block solve is stood in for by numpy on each rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2310_03341_b300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _blocks():
    rng = np.random.default_rng(0)
    sizes = [48, 8, 32, 32, 16, 8, 48, 24]
    mats = []
    for n in sizes:
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        mats.append((A + A.conj().T) / 2)
    return sizes, mats


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes, mats = _blocks()
        mine = sharding.partition_blocks(sizes, world)[rank]
        local = {i: np.linalg.eigvalsh(mats[i]) for i in mine}
        spectra = sharding.gather_spectra(local, sizes, world)
        t = sharding.max_over_ranks(1.5 + rank)
        q.put((rank, [s.tolist() for s in spectra], t))
    finally:
        dist.destroy_process_group()


def test_partition_balances_cubic_cost():
    sizes = [4608] * 64 + [2048] * 64 + [1152] * 64 + [512] * 64
    parts = sharding.partition_blocks(sizes, 4)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    loads = [sum(sizes[i] ** 3 for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.02


def test_gather_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes, mats = _blocks()
    ref = [np.linalg.eigvalsh(A) for A in mats]
    for rank, spectra, t in out:
        assert t == 2.5
        for s, r in zip(spectra, ref):
            assert np.allclose(s, r, atol=1e-12)
