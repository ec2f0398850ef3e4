"""Storage order of a scene: the Z-order of its means, taken once at load.

No per-Gaussian result of the method depends on where a Gaussian sits in
the arrays (only the order of floating-point sums into an atlas voxel
does), so a scene can be stored in whatever order suits the device: in the
Z-order of the means, consecutive receivers are neighbours in direction from
any light and the attenuation's atlas taps of a warp share sectors.  Parts
that must stay contiguous (an avatar, each object of a crowd) are ordered
within themselves.  The permutation comes from ``dgsm_spatial_order``.
"""
from __future__ import annotations

import numpy as np

from . import scenes


def zorder_permutation(nat, means: np.ndarray, bounds, device) -> np.ndarray:
    """The permutation (host int64) that Z-orders each part [bounds[i],
    bounds[i+1]) of `means` within itself (parts keep their places)."""
    import torch
    perm = np.arange(means.shape[0], dtype=np.int64)
    for b0, b1 in zip(bounds[:-1], bounds[1:]):
        if b1 - b0 > 1:
            m = torch.as_tensor(np.ascontiguousarray(means[b0:b1])).to(device)
            perm[b0:b1] = b0 + nat.dgsm_spatial_order(m).cpu().numpy().astype(np.int64)
    return perm


def zorder_scene(nat, sc: scenes.Scene, bounds, device) -> tuple[scenes.Scene, np.ndarray]:
    """`sc` stored in the Z-order of its means within each part (see
    zorder_permutation), its meta kept; returns (scene, permutation)."""
    perm = zorder_permutation(nat, sc.means, bounds, device)
    out = scenes.subset(sc, perm)
    out.meta = dict(sc.meta)
    out.meta["order"] = "z-order of the means within each part"
    return out, perm


def room_parts(sc: scenes.Scene):
    """Part bounds of a room workload's scene: the room, then its avatar."""
    av = sc.meta.get("avatar")
    if av is None:
        return [0, sc.n]
    return sorted({0, int(av.start), int(av.stop), sc.n})
