"""Host logic of the multi-process (one process per GPU) path.

A gradient step on one scan (Sec. 3, Eq. 1-2) has no exchange between
processes when every process owns a whole scan: each rank runs its own
replica and the job's throughput is the units all ranks processed over the
slowest rank's time.  The frame-sharded alternative (one scan's frames spread
over ranks) would sum the per-frame adjoint contributions of Eq. 2 with one
all-reduce of the volume gradient and keep each frame's pose update local; the
helpers below give its contiguous frame partition so that the partition can be
checked on CPU ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def frame_ranges(n_frames: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, balanced [begin, end) frame ranges, one per rank (sizes differ by <= 1)."""
    if n_frames < 0 or world < 1:
        raise ValueError("need n_frames >= 0 and world >= 1")
    base, extra = divmod(n_frames, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def max_over_ranks(x: float, device: torch.device | str = "cpu") -> float:
    """The largest `x` over the ranks of the default process group (x itself when alone).

    `device` must be one the group's backend accepts: a CUDA device for NCCL, the
    CPU for gloo."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    if seconds <= 0:
        raise ValueError("seconds must be positive")
    return world * units_per_rank / seconds
