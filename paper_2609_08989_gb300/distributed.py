"""Sharding one camera over several GPUs (one process per GPU).

Rays are independent, so an image splits into contiguous pixel ranges, one per
rank, traced with the C ABI's pix_begin / pix_count; there is no exchange
during tracing.  The only collective is an optional gather of the finished
per-rank outputs (host side, any torch.distributed backend).  Ranges are
balanced by pixel count; ``weights`` (e.g. a previous image's step counts)
balance them by expected work instead.
"""
from __future__ import annotations

from typing import Callable, Dict, Optional, Sequence, Tuple

import numpy as np

FIELDS_1D = ("code", "n_cross", "intensity", "h_max", "steps", "rejects")
FIELDS_2D = ("r_cross", "g", "I_cross")


def pixel_range(npix: int, rank: int, world: int, weights: Optional[np.ndarray] = None,
                align: int = 1) -> Tuple[int, int]:
    """[begin, begin + count) of the rank's share of npix pixels.  align: the
    interior cuts fall on multiples of it (e.g. 4 camera rows, so that every
    range is traced in the tracer's 8 x 4 pixel tiles)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    if align < 1:
        raise ValueError("align must be >= 1")
    if weights is None:
        if align == 1:
            base, extra = divmod(npix, world)
            begin = rank * base + min(rank, extra)
            return begin, base + (1 if rank < extra else 0)
        w = np.ones(npix)
    else:
        w = np.asarray(weights, dtype=np.float64)
    if w.shape != (npix,) or np.any(w < 0):
        raise ValueError("weights must be npix non-negative numbers")
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    cuts = [int(np.searchsorted(cum, total * k / world, side="left")) for k in range(world + 1)]
    cuts = [min(npix, align * int(round(c / align))) for c in cuts]
    cuts[0], cuts[-1] = 0, npix
    for k in range(1, world + 1):
        cuts[k] = max(cuts[k], cuts[k - 1])
    return cuts[rank], cuts[rank + 1] - cuts[rank]


def trace_shard(trace: Callable[..., Dict[str, np.ndarray]], scene, rank: int, world: int,
                weights: Optional[np.ndarray] = None, align: int = 1) -> Tuple[int, Dict[str, np.ndarray]]:
    """Trace this rank's pixel range with ``trace(scene, pix_begin, pix_count)``."""
    begin, count = pixel_range(scene.nx * scene.ny, rank, world, weights, align)
    return begin, trace(scene, begin, count)


def gather_image(begin: int, out: Dict[str, np.ndarray], npix: int, group=None) -> Optional[Dict[str, np.ndarray]]:
    """Assemble the full image on rank 0 from every rank's (begin, outputs)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    pieces = [None] * world
    dist.all_gather_object(pieces, (begin, {k: np.asarray(v) for k, v in out.items()}), group=group)
    if dist.get_rank(group) != 0:
        return None
    full = {}
    for k in FIELDS_1D:
        full[k] = np.zeros(npix, dtype=pieces[0][1][k].dtype)
    for k in FIELDS_2D:
        full[k] = np.zeros((3, npix), dtype=pieces[0][1][k].dtype)
    for b, o in pieces:
        n = len(o["code"])
        for k in FIELDS_1D:
            full[k][b:b + n] = o[k]
        for k in FIELDS_2D:
            full[k][:, b:b + n] = o[k]
    return full
