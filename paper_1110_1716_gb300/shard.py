"""Sharding of one scan over ranks (one process per GPU).

The scan has no data-path exchange when each rank owns a slice of the
start positions and reads past its end (lazy data partitioning, Sec. III.D.2):
rank r reports exactly the matches whose start lies in its slice, so the union
over ranks is the full match set. These helpers split the work and combine
the results and timings over a torch.distributed process group.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def start_slice(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[lo, hi) of the starts rank `rank` owns among n positions."""
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi


def gather_matches(matches: np.ndarray, group=None) -> np.ndarray:
    """All ranks' (k, w) uint32 match rows, concatenated on every rank
    (variable sizes: lengths first, then padded rows)."""
    import torch
    import torch.distributed as dist
    m = np.ascontiguousarray(matches, dtype=np.uint32)
    w = m.shape[1] if m.ndim == 2 else 3
    world = dist.get_world_size(group)
    k = torch.tensor([m.shape[0]], dtype=torch.int64)
    ks = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(ks, k, group=group)
    kmax = max(int(x.item()) for x in ks)
    buf = torch.zeros((kmax, w), dtype=torch.int64)
    if m.shape[0]:
        buf[:m.shape[0]] = torch.from_numpy(m.astype(np.int64))
    bufs = [torch.zeros((kmax, w), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    parts = [b[:int(kk.item())].numpy() for b, kk in zip(bufs, ks)]
    return np.concatenate(parts).astype(np.uint32) if parts else np.zeros((0, w), np.uint32)


def max_over_ranks(value: float, group=None) -> float:
    """The largest `value` over all ranks (step times: the job takes as long
    as its slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_throughput(bytes_per_rank: int, world: int, step_s_max: float) -> float:
    """Whole-job bytes per second: every rank's bytes over the slowest rank's
    step time (weak scaling: each rank scans its own text)."""
    return bytes_per_rank * world / step_s_max
