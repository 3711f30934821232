"""Host-side helpers of the multi-GPU (data-parallel) mode.

Instances are independent, so the path shards by instance: one batch is
split into per-rank shards by estimated cost (longest processing time first,
partition_lpt), each rank runs its shard as its own batch, and no collective
enters the unrolled path.  Two exchanges remain: the timing of a
benchmark step is the slowest rank's (maximum over ranks), and a training
step sums the gradients of the parameters every instance shares (the
per-step log rho_k / alpha_k, the hyperparameter policy, the warm-start
network) over the ranks' instances.  Both run through torch.distributed on
whatever backend the process group uses (NCCL on GPUs, gloo on CPU).
"""
import heapq

import numpy as np
import torch
import torch.distributed as dist

_PSD = 4   # cone code of the PSD cone (the C ABI's)


def _active():
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank scalar over all ranks (the value itself
    without a multi-rank process group)."""
    if not _active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def sum_gradients(params) -> None:
    """Sum the .grad of each parameter over the ranks in place: the gradient
    of the meta-loss summed over every rank's instances."""
    if not _active():
        return
    for p in params:
        if p.grad is not None:
            dist.all_reduce(p.grad, op=dist.ReduceOp.SUM)


def instance_cost(problem, cg_iters=None) -> float:
    """Estimated work of one instance per unrolled step: the eigensolver's
    sum of p^3 over its PSD blocks, plus the matrix-free CG's traffic, the
    nonzeros of A, A' and P (and the vectors) times the CG iterations per
    solve.  An instance whose reduced matrix is diagonal for every rho (P
    diagonal, at most one nonzero per row of A) is solved in one step; others
    take cg_iters (default 50)."""
    psd = sum(float(d) ** 3 for (t, d) in problem.cones if t == _PSD)
    A, P = problem.A.tocsr(), problem.P.tocsr()
    diag_P = P.nnz == 0 or (P.nnz == np.count_nonzero(P.diagonal()) and P.nnz <= P.shape[0])
    one_per_row = A.shape[0] == 0 or int(np.diff(A.indptr).max()) <= 1
    its = 1.0 if (diag_P and one_per_row) else float(50 if cg_iters is None else cg_iters)
    return psd + its * (2 * A.nnz + P.nnz + 2 * problem.n + problem.m)


def partition_lpt(costs, world):
    """Longest processing time first: instances in decreasing cost (ties: the
    lower index first) go to the rank with the least total so far (ties: the
    lower rank).  Returns per-rank lists of instance indices in increasing
    order; the largest rank total is at most 4/3 of the optimum (Graham)."""
    costs = [float(c) for c in costs]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(sh) for sh in shards]


def shard(problems, rank, world, cg_iters=None):
    """This rank's share of one batch: (indices, problems) by partition_lpt."""
    idx = partition_lpt([instance_cost(p, cg_iters) for p in problems], world)[rank]
    return idx, [problems[i] for i in idx]
