"""Host-side multi-rank logic of bench.py on CPU: two gloo ranks, each a
replica, agree on the max of their timings (the value bench.py reports for
N > 1).  No GPU and no collective in the data path are involved."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist = bench.init_dist(w, use_cuda=False)
    mine = 10.0 + 7.5 * rank
    got = bench.max_over_ranks(dist, mine)
    dist.barrier()
    q.put((rank, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 17.5, 1: 17.5}


def test_single_rank_has_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1, use_cuda=False) is None
    assert bench.max_over_ranks(None, 3.25) == 3.25
