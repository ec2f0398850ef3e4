"""Host-side sharding of the hot path over ranks (one process per GPU).

Lights are independent problems (one atlas per light, Sec. 3.2), so ranks
split the lights and need no exchange on the data path.  Only the
benchmark's timing and unit counts are reduced across ranks.
"""
from __future__ import annotations

import numpy as np


def lights_for_rank(lights: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Round-robin share of the (L,3) light array for `rank` (may be empty)."""
    lights = np.ascontiguousarray(lights, dtype=np.float32).reshape(-1, 3)
    return np.ascontiguousarray(lights[rank::world])


def offset_light(lights: np.ndarray, rank: int, step: float = 0.25) -> np.ndarray:
    """A distinct light per rank for weak scaling: shift along x by rank*step."""
    out = np.array(lights, dtype=np.float32, copy=True).reshape(-1, 3)
    out[:, 0] += step * rank
    return out


def reduce_step_timing(total_ms: float, units: float, group=None, device=None):
    """(max of total_ms over ranks, sum of units over ranks).

    With no process group (single rank) the inputs are returned as they are.
    """
    import torch
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return float(total_ms), float(units)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
