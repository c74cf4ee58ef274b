"""bench.py's path for N > 1 ranks on the CPU: two gloo ranks (spawned
processes, rendezvous on 127.0.0.1) meet at the barrier, both see the
slowest rank's time, and the whole-job rate counts the units of both ranks
over that time (weak scaling: each rank its own replica)."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = bench.Ranks(dist, world, "cpu")
        r.barrier()
        seconds = r.max(10.0 + 3.0 * rank)  # the last rank is the slowest
        out.put((rank, seconds, bench.whole_job_rate(1000.0, world, seconds)))
        r.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 13.0 for g in got)
    assert all(g[2] == pytest.approx(2000.0 / 13.0, rel=1e-15) for g in got)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks()
    r.barrier()
    assert r.max(4.5) == 4.5
    assert bench.whole_job_rate(300.0, 1, 2.0) == 150.0
