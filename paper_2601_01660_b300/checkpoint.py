"""Checkpoint and resume of the learned transmittance field's training.

The training state of nf_train is held by the caller: per light the float32
parameters, the two Adam moment vectors and the number of steps taken (which
nf_train's step0 uses for bias correction and to continue the counter-based
voxel sampling).  A checkpoint stores that state, plus optionally the
per-tile fallback mask of the surrogate attenuation, in one flat
little-endian file:

    magic "DGSMNF01" | u32 version = 1 | u32 n_lights | u64 n_params per light
    | u64 step | u64 mask_len (0: no mask)
    | f32 params[n_lights][n_params] | f32 adam_m[...] | f32 adam_v[...]
    | u8 mask[mask_len]

Saving copies the device tensors to the host; loading returns tensors on the
requested device.  Writes go to a temporary file that is renamed into place.
"""
from __future__ import annotations

import os
import struct

import numpy as np
import torch

MAGIC = b"DGSMNF01"
VERSION = 1
_HEADER = struct.Struct("<8sIIQQQ")


def save_field(path: str, params, adam_m, adam_v, step: int, mask=None) -> None:
    """Write the training state (tensors of shape (n_lights, n_params) or
    (n_params,)) and the optional fallback mask (uint8) to `path`."""
    p, m, v = (np.ascontiguousarray(t.detach().cpu().numpy(), dtype="<f4") for t in (params, adam_m, adam_v))
    if p.ndim == 1:
        p, m, v = p[None], m[None], v[None]
    if not (p.shape == m.shape == v.shape) or p.ndim != 2:
        raise ValueError("params and Adam moments must have one shape (n_lights, n_params)")
    mk = np.ascontiguousarray(mask.detach().cpu().numpy(), dtype=np.uint8).ravel() if mask is not None else None
    if step < 0:
        raise ValueError("step must be >= 0")
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(_HEADER.pack(MAGIC, VERSION, p.shape[0], p.shape[1], int(step), 0 if mk is None else mk.size))
        for a in (p, m, v):
            f.write(a.tobytes())
        if mk is not None:
            f.write(mk.tobytes())
    os.replace(tmp, path)


def load_field(path: str, device=None):
    """(params, adam_m, adam_v, step, mask or None) from `path`; tensors of
    shape (n_lights, n_params) on `device` (the mask as uint8)."""
    with open(path, "rb") as f:
        head = f.read(_HEADER.size)
        if len(head) != _HEADER.size:
            raise ValueError(f"{path}: truncated header")
        magic, version, n_lights, n_params, step, mask_len = _HEADER.unpack(head)
        if magic != MAGIC or version != VERSION:
            raise ValueError(f"{path}: not a field checkpoint (magic {magic!r}, version {version})")
        n = n_lights * n_params
        body = f.read(12 * n + mask_len)
        if len(body) != 12 * n + mask_len or f.read(1):
            raise ValueError(f"{path}: size does not match its header")
    arr = np.frombuffer(body[:12 * n], dtype="<f4").reshape(3, n_lights, n_params)
    dev = torch.device(device) if device is not None else torch.device("cpu")
    p, m, v = (torch.from_numpy(arr[i].copy()).to(dev) for i in range(3))
    mask = torch.from_numpy(np.frombuffer(body[12 * n:], dtype=np.uint8).copy()).to(dev) if mask_len else None
    return p, m, v, int(step), mask
