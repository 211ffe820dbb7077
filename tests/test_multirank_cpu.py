"""The replica (N > 1) aggregation of bench.py, and the row-sharded Gram exchange, on CPU ranks over
gloo (world size 2)."""
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


def _sharded_rank(rank, world, port, out):
    """Rank r holds rows r::world of A and B; the Gram and the right-hand side are the all-reduced
    sums of the ranks' partials (the one exchange of a row-sharded basis build)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(11)
    A = rng.standard_normal((90, 13)) / (1.0 + np.arange(13))
    B = rng.standard_normal((90, 2))
    Ap, Bp = A[rank::world], B[rank::world]
    G = torch.from_numpy(Ap.T @ Ap)
    c = torch.from_numpy(Ap.T @ Bp)
    dist.all_reduce(G)
    dist.all_reduce(c)
    out.put((rank, G.numpy(), c.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_gram_and_rhs_all_reduce_to_the_full_problem():
    """A^T A = sum_p A_p^T A_p and A^T B = sum_p A_p^T B_p over row shards: after the all-reduce every
    rank holds the full Gram and right-hand side, and the oracle's basis built from them is the
    unsharded one (the intervals' recursion then needs no further exchange)."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import ihsbin as ob
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(11)
    A = rng.standard_normal((90, 13)) / (1.0 + np.arange(13))
    B = rng.standard_normal((90, 2))
    G, c = A.T @ A, A.T @ B
    for _, Gr, cr in res:
        np.testing.assert_allclose(Gr, G, rtol=1e-13, atol=1e-13 * np.abs(G).max())
        np.testing.assert_allclose(cr, c, rtol=1e-13, atol=1e-13 * np.abs(c).max())
    S = rng.standard_normal((40, 90)) / np.sqrt(40)
    GS = (S @ A).T @ (S @ A)
    P = ob.precond(GS, 0.2)
    full = ob.basis(lambda V: G @ V, P, c, 0.9, 8)
    shard = ob.basis(lambda V: res[1][1] @ V, P, res[1][2], 0.9, 8)
    assert np.max(np.abs(shard - full)) <= 1e-11 * np.max(np.abs(full))
