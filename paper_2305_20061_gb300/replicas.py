"""Multi-GPU execution of the path tracer as independent replicas.

The paths of a frame are independent (counter-based Philox streams keyed by
pixel, sample and vertex), so N GPUs render N disjoint sample ranges of the
same frame with no exchange on the data path.  This module holds the little
host logic around that: which samples a rank renders, the max-over-ranks
timing of a step, and (outside any timed step) the average of the ranks'
images, which equals a single render with N times the samples.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def first_sample(rank: int, world: int, spp: int, frame: int = 0) -> int:
    """First Philox sample index of rank `rank`: frame f, rank r renders samples
    [(f * world + r) * spp, (f * world + r + 1) * spp)."""
    if not (0 <= rank < world) or spp < 1 or frame < 0:
        raise ValueError("bad rank / world / spp / frame")
    return (frame * world + rank) * spp


def max_over_ranks(value: float, device) -> float:
    """The largest of the ranks' values (step times); the value itself without a process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def average_images(img: torch.Tensor) -> torch.Tensor:
    """Mean of the ranks' images (each the mean of its own samples, all ranks the
    same spp): the image of all ranks' samples together.  Every rank gathers all
    partial images, promotes them to FP64 and adds them in rank order before the
    one division and the cast back, so the result is the same on every rank and
    does not depend on the collective's reduction order.  In place; returns img."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        world = dist.get_world_size()
        parts = [torch.empty_like(img) for _ in range(world)]
        dist.all_gather(parts, img.contiguous())
        acc = torch.zeros(img.shape, dtype=torch.float64, device=img.device)
        for p in parts:                     # rank order
            acc += p.to(torch.float64)
        img.copy_((acc / world).to(img.dtype))
    return img
