"""Sharding of one image's sources across ranks.

Rays are independent (Sec. 3.5), so a frame's sources split into contiguous
ranges, one per rank; each rank renders its range with the global source
indices (pivbos_render_range), and the int64 fixed-point partial images sum
-- in any order, exactly -- to the single-GPU image.  The sum is the only
exchange of the data path.
"""
from __future__ import annotations


def source_range(n_sources: int, world: int, rank: int):
    """Contiguous [first, first + count) block of rank `rank` of `world`;
    blocks differ in size by at most one source and cover all sources."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n_sources), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def allreduce_image(image, group=None):
    """Sum an int64 image over all ranks of the default process group."""
    import torch.distributed as dist
    dist.all_reduce(image, op=dist.ReduceOp.SUM, group=group)
    return image
