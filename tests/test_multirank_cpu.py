"""The N > 1 path of the benchmark on CPU with gloo, two ranks: replicas take disjoint
camera sets, times are reduced to the slowest rank, and a rank that leaves before a
collective makes the other fail within the process-group timeout instead of hanging."""
import datetime
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=30):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))


def _replicas(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port)
    cams = list(range(10))
    mine = bench.shard_cameras(cams, rank, world)
    # rank r "measures" r + 1 ms and 20 - r ms
    mx = bench.reduce_max([rank + 1.0, 20.0 - rank], world)
    dist.barrier()
    out.put((rank, mine, mx))
    dist.destroy_process_group()


def _leaver(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port, timeout_s=5)
    if rank == 1:
        out.put((rank, "left"))
        return                      # leaves before the timing collective
    try:
        bench.reduce_max([1.0], world)
        out.put((rank, "no error"))
    except Exception as e:          # gloo reports the lost peer or the timeout
        out.put((rank, "error: " + type(e).__name__))


def _run(fn, world=2, timeout=120):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=fn, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=timeout) for _ in range(world)]
    for p in procs:
        p.join(timeout=timeout)
        if p.is_alive():
            p.kill()
    return sorted(res, key=lambda x: x[0])


def test_two_replicas_shard_cameras_and_reduce_to_the_slowest_rank():
    res = _run(_replicas)
    (r0, c0, m0), (r1, c1, m1) = res
    assert c0 == [0, 2, 4, 6, 8] and c1 == [1, 3, 5, 7, 9]
    assert m0 == m1 == [2.0, 20.0]
    sys.path.insert(0, ROOT)
    import bench
    # whole-job value: both ranks' pixels over the slowest rank's time
    assert bench.whole_job_mpix_s(2, 5, 1_000_000, 100.0) == pytest.approx(100.0)


def test_a_rank_that_leaves_fails_the_collective_instead_of_hanging():
    res = _run(_leaver, timeout=90)
    assert res[1][1] == "left"
    assert res[0][1].startswith("error"), res[0]
