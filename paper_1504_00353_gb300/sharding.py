"""Frame sharding across GPUs of one node (one process per GPU).

Frames are independent (each is its own Fast-SSC decode), so a batch splits
into contiguous frame ranges, one per rank, with no data exchange. The only
collectives are the timing barrier and the max of the per-rank times, which
work over NCCL (GPU tensors) or gloo (CPU tensors).
"""
from __future__ import annotations


def frame_range(n_frames: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of the frames rank `rank` of `world` decodes; the first
    n_frames % world ranks take one extra frame."""
    if world < 1 or not 0 <= rank < world or n_frames < 0:
        raise ValueError("bad rank/world/n_frames")
    base, extra = divmod(n_frames, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device: str = "cpu") -> float:
    """Max of a per-rank scalar over the default process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: str = "cpu") -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
