"""Multi-rank host logic on CPU with gloo (world_size 2): the bench's rank
seeding, max-over-ranks timing and whole-job value, and one step of the
library's pair sharding as far as it runs without a GPU -- each rank keeps
the oracle's I(i, j) entries that lingam_shard_owner gives it, forms partial
M and error sums, and exchanges them the way the sharded ordering's
all-reduce callback must (gather, add in rank order, identical on every
rank); the replicated argmax then matches the single-rank step.  The GPU
form of the same exchange is tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, I, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # bench: per-rank seeds differ, the slowest rank's time sets the job time
        seed = bench.rank_seed(1003, rank)
        t = bench.max_over_ranks(100.0 + 50.0 * rank, world)
        val = bench.job_throughput(1e12, world, 3, t)
        # sharded scoring of one step: rank r keeps the entries the library's
        # ownership gives it (a partition of the off-diagonal pairs)
        import paper_2403_03772_gb300 as pkg
        p = I.shape[0]
        part = np.zeros(2 * p)
        for i in range(p):
            for j in range(p):
                if i != j and pkg.shard_owner(i, j, p, world) == rank:
                    part[i] += min(0.0, I[i, j]) ** 2
                    part[p + i] += 1.0                 # stands in for the error sums
        # the exchange contract: sums identical bit for bit on every rank
        gathered = [torch.zeros(2 * p, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(part))
        total = np.zeros(2 * p)
        for g in gathered:
            total += g.numpy()
        M = -total[:p]
        assert np.all(total[p:] == p - 1)               # every entry counted once
        best = max(range(p), key=lambda a: (M[a], -a))
        out.put((rank, seed, t, val, best, M.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import gen
    import oracle
    ds = gen.cfg1(n=600, d=8)
    step = oracle.search_step(ds.X)
    I = step["I"]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, I, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    res.sort()
    (_, s0, t0, v0, b0, M0), (_, s1, t1, v1, b1, M1) = res
    assert s0 != s1
    assert t0 == t1 == 150.0
    assert v0 == v1 == pytest.approx(1e12 * 2 * 3 / 0.150)
    assert b0 == b1 == step["m_pos"]
    # the all-reduced scores equal the single-rank k_list up to summation order
    assert np.allclose(M0, step["k_list"], rtol=1e-12, atol=1e-15)
    assert M0 == M1
