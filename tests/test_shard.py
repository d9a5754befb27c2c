"""The multi-rank path on CPU: two gloo ranks split a frame into bands and a view batch
into per-rank views, and reduce timings and sample counts the way the benchmark does."""
import os
import socket

import pytest

from paper_1212_3333_gb300 import shard


@pytest.mark.parametrize("height,world", [(0, 1), (1, 2), (7, 3), (2048, 2), (2048, 8), (5, 8)])
def test_bands_cover_the_frame_once(height, world):
    rows = []
    for r in range(world):
        r0, n = shard.band_rows(height, r, world)
        assert n >= 0
        rows.extend(range(r0, r0 + n))
    assert rows == list(range(height))
    sizes = [shard.band_rows(height, r, world)[1] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def test_views_are_partitioned():
    got = sorted(v for r in range(3) for v in shard.views_for_rank(64, r, 3))
    assert got == list(range(64))
    with pytest.raises(ValueError):
        shard.band_rows(10, 2, 2)


def test_reductions_without_a_group_are_identity():
    assert shard.all_max(3.5) == 3.5 and shard.all_sum(2.0) == 2.0
    assert shard.throughput(10.0, 2.0) == (10.0, 2.0, 5.0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r0, n = shard.band_rows(1000, rank, world)
        bands = [None] * world
        dist.all_gather_object(bands, (r0, n))
        views = [None] * world
        dist.all_gather_object(views, shard.views_for_rank(10, rank, world))
        # rank r renders 100 (r + 1) samples in (r + 1) / 10 s
        total, slowest, rate = shard.throughput(100.0 * (rank + 1), 0.1 * (rank + 1))
        shard.barrier()
        q.put((rank, bands, views, total, slowest, rate, shard.all_max(-rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

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
    for rank, bands, views, total, slowest, rate, mx in out:
        assert bands == [(0, 500), (500, 500)]
        assert views == [[0, 2, 4, 6, 8], [1, 3, 5, 7, 9]]
        assert total == 300.0 and slowest == pytest.approx(0.2) and rate == pytest.approx(1500.0)
        assert mx == 0.0
