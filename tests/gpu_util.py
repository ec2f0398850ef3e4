"""Helpers shared by the GPU tests: move seeded scenes to the device."""
import numpy as np
import torch


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def scene_to_dev(sc):
    return {k: dev(getattr(sc, k)) for k in ("means", "scales", "quats", "opac", "colors")}


def texel_sample(rng, L, H, W, n):
    flat = rng.choice(L * H * W, size=min(n, L * H * W), replace=False)
    l, rem = np.divmod(flat, H * W)
    i, j = np.divmod(rem, W)
    return np.stack([l, i, j], 1).astype(np.int32)
