"""The multi-rank (data-parallel) host logic on CPU with two gloo ranks:
disjoint per-rank shards of a workload, the slowest rank's timing, and the
gradient of the parameters shared by every instance summed over the ranks
(here the closed-loop policy's, from the oracle) equal to the gradient of
the whole batch in one process."""
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


def _problems(rank, per_rank=2):
    from synth import maxcut_problem, random_graph_batch
    return [maxcut_problem(nv, e) for nv, e in random_graph_batch(per_rank, 9100 + rank * per_rank, 4, 7, 0.4, 0.6)]


def _params():
    from oracle import policy as op
    rng = np.random.default_rng(2)
    return (rng.standard_normal(op.n_params(op.NF_RHO)) * 0.1, rng.standard_normal(op.n_params(op.NF_ALPHA)) * 0.1,
            op.default_l0())


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle import policy as op
        from paper_2606_13825_b300.dist import max_over_ranks, sum_gradients
        # per-rank shards of the bench workloads do not overlap
        seeds = torch.tensor([bench.SEED0 + rank * bench.N_INST], dtype=torch.int64)
        allseeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(allseeds, seeds)
        # the step time reported is the slowest rank's
        slowest = max_over_ranks(10.0 + rank)
        # shared-parameter gradients: each rank its own instances, then summed
        tr, ta, l0 = _params()
        g = [np.zeros_like(tr), np.zeros_like(ta), np.zeros(5)]
        for pr in _problems(rank):
            _, (a, b, c), _ = op.loss_and_grads(pr, tr, ta, l0, 3)
            g[0] += a
            g[1] += b
            g[2] += c
        params = [torch.nn.Parameter(torch.zeros(v.size, dtype=torch.float64)) for v in g]
        for p, v in zip(params, g):
            p.grad = torch.tensor(v)
        sum_gradients(params)
        if rank == 0:
            out.put(([int(s) for s in allseeds], slowest, [p.grad.numpy().copy() for p in params]))
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
    seeds, slowest, grads = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    from oracle import policy as op
    assert seeds == [bench.SEED0, bench.SEED0 + bench.N_INST]   # shards of N_INST instances, disjoint
    assert slowest == 11.0
    tr, ta, l0 = _params()
    ref = [np.zeros_like(tr), np.zeros_like(ta), np.zeros(5)]
    for rank in range(world):
        for pr in _problems(rank):
            _, (a, b, c), _ = op.loss_and_grads(pr, tr, ta, l0, 3)
            ref[0] += a
            ref[1] += b
            ref[2] += c
    for got, want in zip(grads, ref):
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14)
