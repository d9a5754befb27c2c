"""Sharding across ranks (one process per GPU) and the host-side reductions around it.

Pixels are independent (Sec. 3.3: one ray per pixel), so a frame splits into image-space
bands rendered through `amr_render_params.row0 / rows`, and a batch of views splits into
whole views per rank; either way no rank reads another's data while rendering.  The only
collectives are over scalars: the slowest rank's elapsed time and the total sample count,
which give whole-job throughput.  Works with the NCCL backend (CUDA tensors) and gloo
(CPU tensors); with no process group, or one rank, every reduction is the identity.
"""
from __future__ import annotations

from typing import List, Tuple


def band_rows(height: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous band of image rows for `rank`: (row0, rows), sizes differing by at most
    one, bands in rank order covering [0, height) exactly once.  rows may be 0 when
    height < world."""
    if world < 1 or not 0 <= rank < world or height < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, height >= 0")
    base, extra = divmod(height, world)
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


def views_for_rank(n_views: int, rank: int, world: int) -> List[int]:
    """Round-robin assignment of view indices to ranks."""
    if world < 1 or not 0 <= rank < world or n_views < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_views >= 0")
    return list(range(rank, n_views, world))


def _group():
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return None
    return dist


def _reduce(x: float, op_name: str) -> float:
    dist = _group()
    if dist is None:
        return float(x)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def all_max(x: float) -> float:
    """Maximum of x over the ranks."""
    return _reduce(x, "MAX")


def all_sum(x: float) -> float:
    """Sum of x over the ranks."""
    return _reduce(x, "SUM")


def barrier() -> None:
    dist = _group()
    if dist is not None:
        dist.barrier()


def throughput(samples_local: float, elapsed_s_local: float) -> Tuple[float, float, float]:
    """Whole-job throughput: (total samples, slowest rank's seconds, samples per second)."""
    total = all_sum(samples_local)
    slowest = all_max(elapsed_s_local)
    return total, slowest, (total / slowest if slowest > 0 else 0.0)
