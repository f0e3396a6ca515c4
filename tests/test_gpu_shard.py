"""Pair sharding of one ordering (lingam_set_shard) on one GPU.

Each rank owns a slice of the unordered pair space (lingam_shard_owner);
its context computes pair moments and score terms only for that slice and,
after every step's scoring, hands the partial M and error sums to an
all-reduce callback.  On one GPU the ranks are separate contexts; their
kernels never wait on one another (the exchange waits on the host):

- the ranks' partial first-step scores add up to the unsharded scores;
- R = 2 and 3 ranks as host threads exchanging through a barrier give the
  unsharded order, equal to the FP64 oracle's;
- two processes exchanging over gloo (all-gather, add in rank order) give
  the same order on both ranks.
"""
import os
import socket
import threading

import numpy as np
import pytest

import gen
import oracle
from gpu_util import M_ABS, M_REL, read_golden_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg2(datasets):
    return datasets("cfg2")


@pytest.mark.parametrize("R", [2, 3])
def test_partial_first_step_scores_add_up(cfg2, R):
    import torch
    import paper_2403_03772_gb300 as pkg
    X = torch.from_numpy(cfg2.X).to("cuda:0")
    with pkg.Context(0, "mixed") as c:
        _, M = c.step_measures(X)
    total = np.zeros_like(M)
    for r in range(R):
        with pkg.Context(0, "mixed") as c:
            c.set_shard(r, R, lambda buf: None)
            _, Mr = c.step_measures(X)
        total += Mr
    scale = np.max(np.abs(M))
    assert np.max(np.abs(total - M)) <= M_REL * scale + M_ABS


class _Exchange:
    """Host all-reduce for R ranks in one process: every rank posts its
    buffer, then all add the buffers in rank order (identical sums)."""

    def __init__(self, R):
        self.R = R
        self.bufs = [None] * R
        self.barrier = threading.Barrier(R)
        self.calls = [0] * R

    def make(self, r):
        def allreduce(buf):
            self.bufs[r] = buf.copy()
            self.barrier.wait(timeout=120)
            total = np.zeros_like(buf)
            for q in range(self.R):
                total += self.bufs[q]
            self.barrier.wait(timeout=120)   # all have read before the next step posts
            buf[:] = total
            self.calls[r] += 1
        return allreduce


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("R", [2, 3])
def test_sharded_order_in_threads_equals_oracle(cfg2, R, prec):
    import torch
    import paper_2403_03772_gb300 as pkg
    gold, dig = read_golden_order("cfg2")
    assert dig == cfg2.digest()
    X = torch.from_numpy(cfg2.X).to("cuda:0")
    ex = _Exchange(R)
    orders = [None] * R
    errors = []

    def run(r):
        try:
            torch.cuda.set_device(0)
            with pkg.Context(0, prec) as c:
                c.set_shard(r, R, ex.make(r))
                orders[r] = c.causal_order(X)
        except Exception as e:   # reported below
            errors.append(e)
            ex.barrier.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(R)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errors, errors
    for r in range(R):
        assert list(orders[r]) == list(gold)
    # one exchange per FP32-scored step (p > 32): 100 - 32 of the 99 steps
    assert ex.calls == [cfg2.d - 32] * R


def test_sharded_context_refuses_batches_and_histories(cfg2):
    import torch
    import paper_2403_03772_gb300 as pkg
    X = torch.from_numpy(cfg2.X).to("cuda:0")
    with pkg.Context(0, "mixed") as c:
        with pytest.raises(pkg.LingamError):
            c.set_shard(2, 2, lambda b: None)
        c.set_shard(0, 2, lambda b: None)
        with pytest.raises(pkg.LingamError) as e:
            c.causal_order(X, scores=True)
        assert e.value.code == pkg.ERR_ARG
        with pytest.raises(pkg.LingamError) as e:
            c.causal_order_batch([(cfg2.X, None), (cfg2.X, None)])
        assert e.value.code == pkg.ERR_ARG
        c.set_shard(0, 1)                              # unsharded again
        assert list(c.causal_order(X)) == list(oracle.causal_order(cfg2.X))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import gen as g
    import paper_2403_03772_gb300 as pkg
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        ds = g.cfg2()
        X = torch.from_numpy(ds.X).to("cuda:0")

        def allreduce(buf):
            parts = [torch.zeros(buf.size, dtype=torch.float64) for _ in range(world)]
            dist.all_gather(parts, torch.from_numpy(buf.copy()))
            total = np.zeros_like(buf)
            for t in parts:
                total += t.numpy()
            buf[:] = total

        with pkg.Context(0, "mixed") as c:
            c.set_shard(rank, world, allreduce)
            out.put((rank, [int(v) for v in c.causal_order(X)]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_processes_share_one_ordering(cfg2):
    import torch.multiprocessing as mp
    gold, _ = read_golden_order("cfg2")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res[0] == res[1] == [int(v) for v in gold]
