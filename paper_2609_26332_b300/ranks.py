"""Host-side logic of multi-GPU runs (one process per GPU, launched by torchrun).

Every unit of work here is independent: a replica of a single domain, or a share of
a batch of drops.  No data crosses GPUs during the timed work; the only collectives
are the barrier around the timed region and the max-over-ranks of the measured times
(so the reported time is that of the slowest rank).

* ``rank_world``      RANK / WORLD_SIZE / LOCAL_RANK from the launcher's environment
* ``instance_share``  the contiguous share [start, stop) of a global instance list
                      that rank r of w steps, balanced by cell count
* ``max_over_ranks``  all-reduce MAX of a scalar (any backend: gloo on CPU, NCCL on GPU)
"""
import os


def rank_world():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_share(cells, rank, world):
    """Split instances with the given cell counts into `world` contiguous shares of
    nearly equal total cells; returns (start, stop) of `rank`'s share.  Every instance
    belongs to exactly one share; shares are empty only when there are fewer instances
    than ranks."""
    n = len(cells)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    total = float(sum(cells))
    bounds = [0]
    acc = 0.0
    k = 0
    for r in range(1, world):
        target = total * r / world
        while k < n and acc + cells[k] / 2.0 <= target:
            acc += cells[k]
            k += 1
        # keep at least one instance per remaining share when possible
        k = max(k, bounds[-1] + (1 if n - bounds[-1] > world - r else 0))
        k = min(k, n - (world - r) if n >= world else k)
        bounds.append(k)
        acc = float(sum(cells[:k]))
    bounds.append(n)
    return bounds[rank], bounds[rank + 1]


def max_over_ranks(value, dist=None, device="cpu"):
    """The maximum of `value` over all ranks (the value itself without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
