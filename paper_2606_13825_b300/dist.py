"""Host-side helpers of the multi-GPU (data-parallel) mode.

Instances are independent, so each rank owns its own batch and no
collective enters the unrolled path.  Two exchanges remain: the timing of a
benchmark step is the slowest rank's (maximum over ranks), and a training
step sums the gradients of the parameters every instance shares (the
per-step log rho_k / alpha_k, the hyperparameter policy, the warm-start
network) over the ranks' instances.  Both run through torch.distributed on
whatever backend the process group uses (NCCL on GPUs, gloo on CPU).
"""
import torch
import torch.distributed as dist


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
