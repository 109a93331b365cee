"""Host logic of the multi-GPU form: independent replicas, one per rank.

A single instance is not domain-decomposed, so N GPUs run N independent, differently seeded
instances of the same workload (weak scaling) with no data-path collective.  Ranks meet only
to time the run: a barrier on both sides of the timed region, then the maximum of the
per-rank times and the sum of the per-rank work, so that throughput = all ranks' work / the
slowest rank's time.  Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def init_process_group(backend: str, timeout_s: float = 600.0):
    """Join the job's process group (RANK, WORLD_SIZE, MASTER_ADDR/PORT from the environment)
    with a bounded wait: when a rank fails or never arrives, the next collective of the
    others ends with an error after at most `timeout_s` seconds instead of waiting forever."""
    import datetime

    import torch.distributed as dist
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=float(timeout_s)))
    return dist


def instance_seed(rank: int) -> int:
    """Seed of the initial state integrated by `rank` (rank 0 runs the seed-0 workload)."""
    return int(rank)


def batch_instance_seed(rank: int, i: int) -> int:
    """Seed of instance i of the batch integrated by `rank`."""
    return 1 + int(i) + 1000 * int(rank)


def combine(dist, ms: float, work: float, device="cpu"):
    """(max over ranks of `ms`, sum over ranks of `work`); the inputs unchanged without a
    process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(work)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
