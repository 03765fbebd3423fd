"""Multi-process plumbing for the residual render: roots are independent, so
a render shards by root ranges (one range per rank, no data exchange while
rendering) and the residual images are summed once at the end; timings take
the maximum over ranks.  torch.distributed does the exchange (NCCL on GPUs,
gloo on CPUs)."""
from __future__ import annotations


def shard_roots(n_roots: int, rank: int, world: int) -> tuple[int, int]:
    """Root range [r0, r1) of `rank`: contiguous, disjoint, covering
    [0, n_roots), sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    q, r = divmod(n_roots, world)
    r0 = rank * q + min(rank, r)
    return r0, r0 + q + (1 if rank < r else 0)


def sum_images(img):
    """Sum a residual image over ranks in place (all_reduce SUM)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(img, op=dist.ReduceOp.SUM)
    return img


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a host scalar over ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
