"""bench.py's multi-rank path (one replica per rank, max-over-ranks timing, serving
results gathered to rank 0) on world_size-2 gloo process groups on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w = bench._dist("gloo")
    assert (r, w) == (rank, ws)
    # each rank times its own replica; the reported time is the slowest rank's
    local_ms = 10.0 + 5.0 * rank
    t = bench._max_over_ranks(dist, local_ms, "cpu")
    parts = [None] * ws
    dist.all_gather_object(parts, {"rank": rank, "conv": rank + 1, "lat": [0.1 * (rank + 1)]})
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, parts))


def test_max_over_ranks_and_gather_on_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, parts in res:
        assert t == 15.0                       # max over ranks on every rank
        assert [p["rank"] for p in parts] == [0, 1]
        assert sum(p["conv"] for p in parts) == 3


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    os.environ.pop("WORLD_SIZE", None)
    dist, r, w = bench._dist("gloo")
    assert dist is None and (r, w) == (0, 1)
    assert bench._max_over_ranks(None, 3.5, "cpu") == 3.5
