"""The replica (N > 1) aggregation of bench.py on CPU ranks over gloo (world size 2)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 1 + r seconds for 5 paths; the job time is the slowest rank's
    t = bench.max_over_ranks(1.0 + rank, dist)
    out.put((rank, t, bench.job_throughput(world, 5, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [2.0, 2.0]          # both ranks agree on the slowest time
    assert all(abs(r[2] - 5.0) < 1e-12 for r in res)  # 2 ranks x 5 paths / 2 s


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 10, 2.0) == 5.0
