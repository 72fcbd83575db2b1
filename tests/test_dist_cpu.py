"""The multi-GPU bench path on CPU: two gloo ranks exercise the barrier, the
max-over-ranks timing reduction and the shard split (no GPU, no data-path
collective)."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1007_3818_gb300 import dist
    r, w = dist.init("gloo")
    dist.barrier()
    m = dist.max_over_ranks(0.5 + r)          # each rank's "elapsed time"
    lo, hi = dist.shard(4099, r, w)
    dist.barrier()
    dist.finalize()
    q.put((r, w, m, lo, hi))


def test_two_gloo_ranks_time_max_and_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 1.5 for r in res)  # max over ranks seen by every rank
    spans = [(r[3], r[4]) for r in res]
    assert spans[0][0] == 0 and spans[0][1] == spans[1][0] and spans[1][1] == 4099
    assert abs((spans[0][1] - spans[0][0]) - (spans[1][1] - spans[1][0])) <= 1


def test_single_process_helpers_are_identity():
    from paper_1007_3818_gb300 import dist
    assert dist.max_over_ranks(3.25) == 3.25
    assert dist.shard(10, 0, 1) == (0, 10)
