"""The multi-rank driver logic on CPU: two gloo ranks (127.0.0.1) shard units
without overlap or gaps, draw distinct instance sets, and agree on the
maximum of their times."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2306_05789_gb300 import ranks  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = ranks.rank_env()
        lo, hi = ranks.shard_range(257, r, w)
        ranks.barrier()
        t = ranks.max_over_ranks(1.5 + r)
        got = [None] * w
        dist.all_gather_object(got, (lo, hi, ranks.instance_seed(0, r)))
        out.put((r, w, lr, t, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, lr, t, got in res:
        assert w == 2 and lr == r
        assert t == 2.5                      # the max of 1.5 and 2.5 on both ranks
        (lo0, hi0, s0), (lo1, hi1, s1) = got
        assert lo0 == 0 and hi0 == lo1 and hi1 == 257 and abs((hi0 - lo0) - (hi1 - lo1)) <= 1
        assert s0 != s1


def test_shard_range_partitions_any_count():
    for count in (0, 1, 5, 256, 1001):
        for world in (1, 2, 3, 8):
            spans = [ranks.shard_range(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            assert all(spans[k][1] == spans[k + 1][0] for k in range(world - 1))
    with pytest.raises(ValueError):
        ranks.shard_range(4, 2, 2)
