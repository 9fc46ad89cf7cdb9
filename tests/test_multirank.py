"""The multi-rank path on CPU: two gloo ranks shard independent blocks and messages with no
data-path collective; their results, gathered here only to check them, equal one process's."""
import os
import socket

import numpy as np
import pytest

from paper_1506_08503_gb300 import sharding, workloads


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out: dict):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        orc = oracle.oracle()
        w = workloads.plain(5, 3001)
        lo, hi = sharding.block_range(3001, rank, world)
        mine = orc.encrypt_blocks(w.key, w.data[16 * lo:16 * hi], threads=2)
        # gather only to check; the benchmark path has no data collective
        sizes = [None] * world
        dist.all_gather_object(sizes, (lo, hi, mine.tobytes()))
        t = sharding.max_over_ranks(float(rank + 1))
        m = workloads.batched_messages(6, m=64, median=512.0, hi=1 << 16)
        ranges = sharding.message_ranges(m.lengths, world)
        f, l = ranges[rank]
        parts = [orc.encrypt_blocks(m.keys[i], m.data[m.offsets[i]:m.offsets[i] + m.lengths[i]], threads=1)
                 for i in range(f, l)]
        msg_parts = [None] * world
        dist.all_gather_object(msg_parts, (f, l, b"".join(p.tobytes() for p in parts)))
        if rank == 0:
            out.update(blocks=sizes, tmax=t, msgs=msg_parts, seeds=[sharding.weak_scaling_seed(1, r) for r in range(world)])
    finally:
        dist.destroy_process_group()


def _worker(rank, world, port, q):
    out = {}
    _rank_main(rank, world, port, out)
    if rank == 0:
        q.put(out)


def test_two_gloo_ranks_shard_without_collectives():
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    orc = oracle.oracle()
    w = workloads.plain(5, 3001)
    whole = orc.encrypt_blocks(w.key, w.data, threads=2).tobytes()
    ranges = [(lo, hi) for lo, hi, _ in out["blocks"]]
    assert ranges == [(0, 1500), (1500, 3001)]
    assert b"".join(b for _, _, b in out["blocks"]) == whole
    assert out["tmax"] == 2.0
    m = workloads.batched_messages(6, m=64, median=512.0, hi=1 << 16)
    want = b"".join(orc.encrypt_blocks(m.keys[i], m.data[m.offsets[i]:m.offsets[i] + m.lengths[i]], threads=1).tobytes()
                    for i in range(64))
    assert b"".join(b for _, _, b in out["msgs"]) == want
    assert out["seeds"] == [1, 1001]


def test_ranges_cover_exactly_once():
    for n in (0, 1, 7, 1000, 2 ** 26 + 3):
        for world in (1, 2, 3, 8):
            rs = [sharding.block_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1
    lengths = np.array([5, 100, 1, 1, 50, 50, 3])
    for world in (1, 2, 3, 7, 9):
        mr = sharding.message_ranges(lengths, world)
        assert len(mr) == world and mr[0][0] == 0 and mr[-1][1] == len(lengths)
        assert all(a[1] == b[0] for a, b in zip(mr, mr[1:]))
    with pytest.raises(ValueError):
        sharding.block_range(10, 2, 2)
