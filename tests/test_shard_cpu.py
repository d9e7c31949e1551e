"""Multi-GPU host logic on CPU: stream sharding is a partition (every stream on exactly one rank, the same
rank for all of a stream's chunks), and the whole-job aggregate over world_size-2 gloo ranks sums the
units and takes the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2606_04410_b300 import shard as _shard_mod  # noqa: F401  (the module imports no CUDA)


def test_shard_is_a_partition_with_stream_affinity():
    from paper_2606_04410_b300.shard import shard
    ids = list(range(64))
    for world in (1, 2, 3, 8):
        parts = [shard(ids, r, world) for r in range(world)]
        flat = sorted(s for p in parts for s in p)
        assert flat == ids
        for r, p in enumerate(parts):
            assert all(s % world == r for s in p)
    with pytest.raises(ValueError):
        shard(ids, 2, 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2606_04410_b300.shard import aggregate, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(list(range(10)), rank, world)
    units = 8 * len(mine)                 # 8 frames per chunk, one chunk per owned stream
    ms = 100.0 + 50.0 * rank              # rank 1 is the slower one
    dist.barrier()
    tot_units, max_ms = aggregate(units, ms, dist)
    q.put((rank, mine, tot_units, max_ms))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, u0, t0), (r1, m1, u1, t1) = res
    assert sorted(m0 + m1) == list(range(10)) and not set(m0) & set(m1)
    assert u0 == u1 == 80.0
    assert t0 == t1 == 150.0
    assert 80.0 / (150.0 / 1000.0) == pytest.approx(533.333, rel=1e-4)
