"""The bench's replica path on two CPU ranks (gloo): barrier, max-over-ranks
timing and the whole-job aggregate. No GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, loc = bench.dist_env()
    d = bench.Dist(w, loc, "gloo")
    d.barrier()
    t_local = 10.0 + 5.0 * rank  # ms: rank 1 is slower
    t_max = d.max(t_local)
    val = bench.aggregate_rate(w, 1000.0, t_max)
    d.close()
    q.put((r, t_max, val))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for r, t_max, val in out:
        assert t_max == 15.0
        assert abs(val - 2 * 1000.0 / 0.015) < 1e-6
