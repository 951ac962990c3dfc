"""The multi-GPU host logic of bench.py on CPU: two gloo ranks (world size
2) take the maximum of their times and report the whole-job rate, as the
N-replica run does over NCCL."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0 + 50.0 * rank, 300.0 - 10.0 * rank]     # rank 1 is slower, rank 0 slower e2e
    got = bench.max_over_ranks(ms, "cpu")
    out.put((rank, got, bench.job_rate(world, 20, got[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [150.0, 300.0]
        assert abs(rate - 2 * 20 / 0.150) < 1e-9


def test_single_process_needs_no_group():
    assert bench.max_over_ranks([1.5, 2.5], "cpu") == [1.5, 2.5]
    assert bench.job_rate(1, 10, 500.0) == 20.0
