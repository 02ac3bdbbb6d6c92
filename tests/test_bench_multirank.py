"""The multi-GPU launch of bench.py runs one independent replica per rank and
combines them with a max over ranks of the timed region and a sum of the
iterations.  This checks that host logic with two gloo ranks on the CPU
(127.0.0.1 rendezvous), as torchrun would start them."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    dist = bench.dist_init("gloo")
    ws, r, local = bench.dist_env()
    t_max = bench.reduce_max(10.0 + rank, dist)
    n_sum = bench.reduce_sum(1000 * (rank + 1), dist)
    bench.barrier(dist)
    out[rank] = (ws, r, t_max, n_sum)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ws, rr, t_max, n_sum = out[r]
        assert ws == 2 and rr == r
        assert t_max == 11.0  # slowest rank's time
        assert n_sum == 3000  # all ranks' units


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_max(3.5, None) == 3.5
    assert bench.reduce_sum(7, None) == 7.0
    bench.barrier(None)
