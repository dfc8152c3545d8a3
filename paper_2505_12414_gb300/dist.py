"""Multi-rank host logic (torch.distributed): one process per GPU.

The likelihood shards two ways (paper Sec. 1: the per-event terms are independent):
  * independent samples per rank (toys, fits, or the bench's per-rank 1M-event sample):
    no exchange on the data path, only the max-over-ranks step time (weak scaling);
  * events of one sample split across ranks: each rank evaluates its shard and the K
    per-rank sums are added in rank order (a deterministic all-gather, not an all-reduce
    whose summation order is unspecified).
"""
import os

import torch
import torch.distributed as dist


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def sample_stream(rank, base=0):
    """Seed stream of a rank's independent sample (weak scaling)."""
    return base + rank


def max_over_ranks(x, device="cpu"):
    """Maximum of a float over all ranks (the step time of the slowest rank)."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_in_rank_order(values, device="cpu"):
    """Element-wise sum of a float vector over ranks, added in rank order 0, 1, ..."""
    v = torch.as_tensor(values, dtype=torch.float64, device=device).reshape(-1)
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return v.cpu().numpy()
    parts = [torch.empty_like(v) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, v)
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    return total.cpu().numpy()


def shard(n, rank, world):
    """Contiguous event range [lo, hi) of `rank` for an n-event sample split over `world` ranks."""
    return n * rank // world, n * (rank + 1) // world


def whole_job_rate(units_per_rank, world, max_seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / max_seconds
