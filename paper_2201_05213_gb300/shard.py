"""Host-side sharding of a decode batch over ranks (one GPU per rank).

Units (images, their patches and row streams) are independent (Section 3:
pixels of different units never share context), so a batch splits across
GPUs with no data-path collective: each rank decodes a subset of the
containers with its own persistent launch.  This module only plans and
slices; it does no arithmetic of the method.

The plan is longest-processing-time first over an image's decode cost, the
pixel count (the work of every step is split over all SMs, so a rank's time
grows with its pixels; its step count is the largest unit's T, the same for
every rank once images exceed a patch).  Every rank computes the same plan
from the same sizes, so no plan needs to be exchanged.
"""
from __future__ import annotations

import numpy as np


def image_cost(H: int, W: int) -> int:
    """Decode cost of one image (pixels)."""
    return int(H) * int(W)


def plan_shards(sizes, world: int):
    """Images of each rank: LPT over image_cost, ties broken by index.

    sizes: list of (H, W).  Returns `world` sorted lists of image indices that
    together hold every index exactly once.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-image_cost(*sizes[i]), i))
    load = [0] * world
    plan = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        plan[r].append(i)
        load[r] += image_cost(*sizes[i])
    return [sorted(p) for p in plan]


def rank_batch(data, offsets, idx):
    """Containers `idx` of a host batch as one contiguous batch.

    data: uint8 array of concatenated containers; offsets: n+1 int64 byte
    offsets.  Returns (bytes, offsets) of the selected containers in the
    order of idx.  Containers are padded to 16 bytes, so the slices keep the
    16-byte alignment the library requires.
    """
    data = np.asarray(data, dtype=np.uint8)
    offsets = np.asarray(offsets, dtype=np.int64)
    parts, offs = [], [0]
    for i in idx:
        a, b = int(offsets[i]), int(offsets[i + 1])
        if a % 16 or b % 16:
            raise ValueError("container offsets must be multiples of 16")
        parts.append(data[a:b])
        offs.append(offs[-1] + (b - a))
    out = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    return out, np.asarray(offs, dtype=np.int64)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (the
    timing reduction of a multi-GPU run); the value itself when not
    distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])
