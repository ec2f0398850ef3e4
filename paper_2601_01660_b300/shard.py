"""Host-side sharding of the hot path over ranks (one process per GPU).

Lights are independent problems (one atlas per light, Sec. 3.2), so ranks
split the lights and need no exchange on the data path.  Only the
benchmark's timing and unit counts are reduced across ranks.  When there are
fewer lights than ranks, one light set's atlas can be split by rows instead:
each rank builds a band of whole tile rows (every rank bins all Gaussians)
and one all-gather of the bands gives every rank the full atlas.
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


# ---- one light's atlas split over ranks (bands of whole tile rows) ----------

def band_rows(H: int, tile: int, rank: int, world: int):
    """(row0, row1, band height) of `rank`'s band of an H-row atlas: whole
    tile rows, ceil(tile rows / world) of them per rank (the last bands may be
    shorter or empty); the band height pads every band to one size for the
    all-gather."""
    tile_rows = -(-H // tile)
    per = -(-tile_rows // world)
    r0 = min(rank * per * tile, H)
    r1 = min((rank + 1) * per * tile, H)
    return r0, r1, per * tile


def banded_atlas(build_band, extract, insert, empty, H: int, tile: int, group=None):
    """The atlas of one light set, each rank building only its band, then one
    all-gather of the (planes, band height, W) slabs, each rank's rows put
    back into the full (planes, H, W) atlas on every rank.

    build_band(row0, row1) -> full-size atlas with those rows built;
    extract(full, row0, rows, slab) copies the band rows into a slab;
    insert(slab, row0, rows, atlas) copies them back; empty(rows) allocates
    a (planes, rows, W) atlas.  With no process group it runs as one rank."""
    import torch.distributed as dist
    grouped = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank(group) if grouped else 0
    world = dist.get_world_size(group) if grouped else 1
    r0, r1, hb = band_rows(H, tile, rank, world)
    slab = empty(hb)
    if r1 > r0:
        extract(build_band(r0, r1), r0, r1 - r0, slab)
    parts = [empty(hb) for _ in range(world)]
    if grouped:
        dist.all_gather(parts, slab, group=group)
    else:
        parts[0] = slab
    atlas = empty(H)
    for p, part in enumerate(parts):
        q0, q1, _ = band_rows(H, tile, p, world)
        if q1 > q0:
            insert(part, q0, q1 - q0, atlas)
    return atlas


def build_banded(nat, means, scales, quats, opac, lights, H, W, radii, params=None, group=None):
    """dgsm_build of one light set split over the ranks of `group` by atlas
    rows: every rank bins all Gaussians, builds its band (dgsm_build_band),
    and the bands are all-gathered (NCCL on GPUs) into the full atlas
    [L][K][H][W] on every rank."""
    import torch
    p = dict(params or {})
    tile = int(p.get("tile", 8))
    L, K = lights.shape[0], radii.shape[0]
    dt = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[int(p.get("atlas_dtype", 0))]
    dev = means.device

    def empty(rows):
        return torch.empty((L, K, rows, W), dtype=dt, device=dev)

    return banded_atlas(
        lambda r0, r1: nat.dgsm_build_band(means, scales, quats, opac, lights, H, W, radii, r0, r1, params=params),
        lambda full, r0, n, slab: nat.dgsm_atlas_rows_copy(full, r0, slab, 0, n),
        lambda slab, q0, n, atlas: nat.dgsm_atlas_rows_copy(slab, 0, atlas, q0, n),
        empty, H, tile, group)
