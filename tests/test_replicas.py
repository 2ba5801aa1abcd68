"""The multi-GPU form of the bench is replicas only (one independent problem per
rank, no data-path collective).  Its host logic -- rank environment, the max of
the per-rank times and the sum of the points over ranks, the per-rank seeds --
runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    w, r, loc = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    ms = 100.0 + 10.0 * r            # a slower rank sets the job time
    points = 1000.0 * (r + 1)
    t = bench.max_over_ranks(dist, ms)
    p = bench.sum_over_ranks(dist, points)
    out.put((r, w, loc, t, p))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_points():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, loc, t, p in res:
        assert w == ws and loc == r
        assert t == 110.0          # max over ranks
        assert p == 3000.0         # total points of all ranks


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    ws, rank, local = bench.dist_env()
    assert (ws, rank, local) == (1, 0, 0)
    assert bench.init_dist(ws, "gloo") is None
    assert bench.max_over_ranks(None, 5.0) == 5.0 and bench.sum_over_ranks(None, 7.0) == 7.0
