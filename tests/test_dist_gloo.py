"""The multi-rank (data-parallel) host logic on CPU with two gloo ranks: one
batch split into per-rank shards by estimated cost (LPT) that are disjoint and
cover the batch, the slowest rank's timing, and the gradient of the
parameters shared by every instance summed over the ranks (here the
closed-loop policy's, from the oracle) equal to the gradient of the whole
batch in one process."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    """One batch of uneven instances (max-cut SDPs of 3..8 vertices)."""
    from synth import maxcut_problem, random_graph_batch
    return [maxcut_problem(nv, e) for nv, e in random_graph_batch(5, 9100, 3, 8, 0.4, 0.6)]


def _params():
    from oracle import policy as op
    rng = np.random.default_rng(2)
    return (rng.standard_normal(op.n_params(op.NF_RHO)) * 0.1, rng.standard_normal(op.n_params(op.NF_ALPHA)) * 0.1,
            op.default_l0())


def _grads(problems):
    from oracle import policy as op
    tr, ta, l0 = _params()
    g = [np.zeros_like(tr), np.zeros_like(ta), np.zeros(5)]
    for pr in problems:
        _, (a, b, c), _ = op.loss_and_grads(pr, tr, ta, l0, 3)
        g[0] += a
        g[1] += b
        g[2] += c
    return g


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_13825_b300.dist import max_over_ranks, sum_gradients, shard
        # this rank's share of the one batch
        idx, mine = shard(_batch(), rank, world)
        allidx = [None] * world
        dist.all_gather_object(allidx, idx)
        # the step time reported is the slowest rank's
        slowest = max_over_ranks(10.0 + rank)
        # shared-parameter gradients: each rank its own instances, then summed
        g = _grads(mine)
        params = [torch.nn.Parameter(torch.zeros(v.size, dtype=torch.float64)) for v in g]
        for p, v in zip(params, g):
            p.grad = torch.tensor(v)
        sum_gradients(params)
        if rank == 0:
            out.put((allidx, slowest, [p.grad.numpy().copy() for p in params]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    allidx, slowest, grads = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2606_13825_b300.dist import instance_cost
    batch = _batch()
    # the shards are disjoint and cover the batch; loads within Graham's 4/3
    flat = sorted(i for sh in allidx for i in sh)
    assert flat == list(range(len(batch))), allidx
    assert all(len(sh) > 0 for sh in allidx)
    cost = [instance_cost(p) for p in batch]
    loads = [sum(cost[i] for i in sh) for sh in allidx]
    assert max(loads) <= 4.0 / 3.0 * max(sum(cost) / world, max(cost)) + 1e-9
    assert slowest == 11.0
    for got, want in zip(grads, _grads(batch)):
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14)


def test_partition_lpt_against_brute_force():
    """LPT on small cost lists: a partition of the indices, deterministic,
    and within Graham's bound (4/3 - 1/(3 world)) of the optimum found by
    trying every assignment; and the rule itself on a case worked by hand."""
    from paper_2606_13825_b300.dist import partition_lpt
    rng = np.random.default_rng(3)
    for _ in range(30):
        n, world = int(rng.integers(1, 8)), int(rng.integers(1, 4))
        cost = list(rng.integers(1, 50, size=n).astype(float))
        sh = partition_lpt(cost, world)
        assert sorted(i for s in sh for i in s) == list(range(n))
        assert sh == partition_lpt(cost, world)
        best = min(max(sum(cost[i] for i in range(n) if a[i] == r) for r in range(world))
                   for a in itertools.product(range(world), repeat=n))
        got = max(sum(cost[i] for i in s) for s in sh)
        assert got <= (4.0 / 3.0 - 1.0 / (3 * world)) * best + 1e-9, (cost, world, sh)
    # costs 3, 7, 4, 3, 5 over two ranks, largest first: 7 (index 1) -> r0,
    # 5 (index 4) -> r1, 4 (index 2) -> r1 (5 < 7), 3 (index 0) -> r0 (7 < 9),
    # 3 (index 3) -> r1 (9 < 10)
    assert partition_lpt([3, 7, 4, 3, 5], 2) == [[0, 1], [2, 3, 4]]


def test_bench_shards_partition_the_global_batch():
    """The benchmark's per-rank shards of the max-cut workload at two ranks
    are disjoint and cover the 512-instance global batch (instance sizes are
    compared, the generator being deterministic)."""
    import bench
    from synth import random_graph_batch
    from paper_2606_13825_b300.dist import partition_lpt, instance_cost
    from synth import maxcut_problem
    graphs = random_graph_batch(bench.N_INST * 2, bench.SEED0, 20, 80, 0.1, 0.5)
    sh = partition_lpt([instance_cost(maxcut_problem(nv, e)) for nv, e in graphs], 2)
    assert sorted(sh[0] + sh[1]) == list(range(2 * bench.N_INST))
    n0 = sum(graphs[i][0] ** 3 for i in sh[0])
    n1 = sum(graphs[i][0] ** 3 for i in sh[1])
    assert abs(n0 - n1) <= 0.01 * (n0 + n1)
