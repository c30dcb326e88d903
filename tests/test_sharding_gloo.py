"""Multi-rank host logic on CPU (gloo, world sizes 2 and 3): block partition,
eigenvalue all-gather of the batched path, the sharded batched driver, and the
benchmark's max-over-ranks timing.  The per-block solve is stood in for by
numpy on each rank."""
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


def _eigh_batch(mats):
    out = []
    for A in mats:
        w, Z = np.linalg.eigh(A)
        out.append((w, Z))
    return out


def _sharded_worker(rank, world, port, q, nblocks):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes, mats = _blocks()
        sizes, mats = sizes[:nblocks], mats[:nblocks]
        built = []

        def make(i):
            built.append(i)
            return mats[i]

        spectra, local = sharding.solve_sharded(sizes, make, _eigh_batch, rank, world)
        # a block claimed by two ranks is refused on every rank alike
        clash = None
        try:
            sharding.gather_spectra({0: np.zeros(sizes[0])}, sizes, world)
        except RuntimeError as e:
            clash = str(e)
        q.put((rank, [s.tolist() for s in spectra], sorted(built),
               {i: float(np.abs(mats[i] @ Z - Z * w).max()) for i, (w, Z) in local.items()},
               clash))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nblocks", [(2, 8), (3, 2)])
def test_solve_sharded_over_gloo_ranks(world, nblocks):
    """Every block is built and solved on exactly one rank, every rank ends with the whole
    spectrum in block order, and a rank that owns no block (3 ranks, 2 blocks) still joins
    the exchange."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q, nblocks))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes, mats = _blocks()
    ref = [np.linalg.eigvalsh(A) for A in mats[:nblocks]]
    built = sorted(i for _, _, b, _, _ in out for i in b)
    assert built == list(range(nblocks))
    least = min(len(b) for _, _, b, _, _ in out)
    assert least == 0 if world > nblocks else least >= 1
    for rank, spectra, b, resid, clash in out:
        assert sorted(resid) == b
        assert all(r < 1e-10 for r in resid.values())
        assert len(spectra) == nblocks
        for s, r in zip(spectra, ref):
            assert np.allclose(s, r, atol=1e-12)
        # every rank claimed block 0 in the second exchange
        assert clash is not None and "exactly one rank" in clash


def _density_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes, mats = _blocks()
        V = 24
        mine = sharding.partition_blocks(sizes, world)[rank]
        n = torch.zeros(V, dtype=torch.float64)
        nu = torch.zeros(V, dtype=torch.complex128)
        for i in mine:                      # a block's contribution: a seeded field of its own
            r = np.random.default_rng(100 + i)
            n += torch.as_tensor(r.random(V))
            nu += torch.as_tensor(r.standard_normal(V) + 1j * r.standard_normal(V))
        sharding.reduce_densities(n, nu)
        q.put((rank, n.numpy().copy(), nu.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_density_sum_over_three_gloo_ranks():
    """Every rank ends with the sum over all blocks, whichever rank accumulated each block."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_density_worker, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes, _ = _blocks()
    n_ref, nu_ref = np.zeros(24), np.zeros(24, dtype=complex)
    for i in range(len(sizes)):
        r = np.random.default_rng(100 + i)
        n_ref += r.random(24)
        nu_ref += r.standard_normal(24) + 1j * r.standard_normal(24)
    for _, n, nu in out:
        assert np.allclose(n, n_ref, rtol=0, atol=1e-12)
        assert np.allclose(nu, nu_ref, rtol=0, atol=1e-12)
