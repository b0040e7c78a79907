"""Host logic of halo-sharded runs, on CPU: the partition of a lattice's rows
into slabs, each slab's storage rows in the lattice, field slicing, the
neighbour ranks, and the transport of the halo messages between gloo ranks
(world sizes 2 and 3, periodic and walled), plus the all-reduce of the
slabs' FP64 totals.  The device side (pack, unpack, the slab step) runs in
the GPU tests."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1608_01906_gb300 import sharding  # noqa: E402


def test_slab_rows_partition():
    for ny, n in ((2048, 2), (2048, 3), (2048, 7), (100, 4), (64, 8), (96, 1)):
        rows = sharding.slab_rows(ny, n)
        assert len(rows) == n
        assert rows[0][0] == 0
        assert sum(r for _, r in rows) == ny
        for (a, ra), (b, _) in zip(rows, rows[1:]):
            assert a + ra == b and b % sharding.TILE_ROWS == 0
        assert min(r for _, r in rows) >= 2 * sharding.HALO
        sizes = [r for _, r in rows[:-1]]
        assert not sizes or max(sizes) - min(sizes) <= sharding.TILE_ROWS
    with pytest.raises(ValueError):
        sharding.slab_rows(60, 8)  # 7 aligned blocks for 8 slabs
    with pytest.raises(ValueError):
        sharding.slab_rows(64, 0)


def test_storage_rows_and_fields():
    # periodic: the halo rows wrap around the lattice
    r = sharding.storage_rows(0, 16, 48, walls=False)
    assert list(r[:4]) == [44, 45, 46, 47] and list(r[4:20]) == list(range(16)) and list(r[20:]) == [16, 17, 18, 19]
    r = sharding.storage_rows(40, 8, 48, walls=False)
    assert list(r[-4:]) == [0, 1, 2, 3]
    # walled: rows outside the lattice stand in as the nearest lattice row
    r = sharding.storage_rows(0, 16, 48, walls=True)
    assert list(r[:4]) == [0, 0, 0, 0] and r[4] == 0 and r[19] == 15
    r = sharding.storage_rows(32, 16, 48, walls=True)
    assert list(r[-4:]) == [47, 47, 47, 47]
    nx, ny = 5, 12
    f = np.arange(nx * ny, dtype=float)
    u = np.stack([f, -f], axis=1)
    rows = sharding.storage_rows(4, 4, ny, walls=False)
    sf = sharding.slab_fields(f, nx, ny, rows)
    assert sf.shape == (12 * nx,)
    assert np.array_equal(sf.reshape(12, nx)[:, 0], rows * nx)
    su = sharding.slab_fields(u, nx, ny, rows)
    assert su.shape == (12 * nx, 2) and np.array_equal(su[:, 1], -sf)


def test_neighbours():
    assert sharding.neighbours(0, 3, walls=False) == (2, 1)
    assert sharding.neighbours(2, 3, walls=False) == (1, 0)
    assert sharding.neighbours(0, 3, walls=True) == (None, 1)
    assert sharding.neighbours(2, 3, walls=True) == (1, None)
    assert sharding.neighbours(0, 1, walls=False) == (0, 0)
    assert sharding.neighbours(0, 1, walls=True) == (None, None)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, walls, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1608_01906_gb300 import sharding as sh

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 72 * 8  # one FP32 message of an 8-wide lattice (pitch 8)
        # message content names its sender and side
        send = [torch.full((n,), 10.0 * rank + 1.0), torch.full((n,), 10.0 * rank + 2.0)]
        recv = [torch.full((n,), -1.0), torch.full((n,), -1.0)]
        sh.exchange_ranks(send, recv, rank, world, walls, dist)
        tot = sh.allreduce_totals([1.0 + rank, 0.5 * rank, 1e-17 * rank], dist)
        q.put((rank, float(recv[0][0]), float(recv[1][0]), bool(torch.all(recv[0] == recv[0][0])),
               bool(torch.all(recv[1] == recv[1][0])), tot.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,walls", [(2, False), (2, True), (3, False), (3, True)])
def test_exchange_between_gloo_ranks(world, walls):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, walls, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lo, hi, lo_whole, hi_whole, tot in res:
        nlo, nhi = sharding.neighbours(rank, world, walls)
        # recv lo holds the lower slab's send hi; recv hi the upper's send lo
        assert lo == (-1.0 if nlo is None else 10.0 * nlo + 2.0)
        assert hi == (-1.0 if nhi is None else 10.0 * nhi + 1.0)
        assert lo_whole and hi_whole
        assert tot[0] == sum(1.0 + r for r in range(world))
        assert tot[1] == sum(0.5 * r for r in range(world))


def test_single_periodic_rank_is_its_own_neighbour():
    import torch

    send = [torch.tensor([1.0, 2.0]), torch.tensor([3.0, 4.0])]
    recv = [torch.zeros(2), torch.zeros(2)]
    sharding.exchange_ranks(send, recv, 0, 1, False, dist=None)
    assert recv[0].tolist() == [3.0, 4.0] and recv[1].tolist() == [1.0, 2.0]
    recv = [torch.zeros(2), torch.zeros(2)]
    sharding.exchange_ranks(send, recv, 0, 1, True, dist=None)
    assert recv[0].tolist() == [0.0, 0.0] and recv[1].tolist() == [0.0, 0.0]
