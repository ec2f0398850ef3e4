"""FP64 oracle of the per-frame mechanics around the method for moving
avatars: rigid motion of whole objects, per-object alpha-weighted centroids,
and attenuation by a static atlas times a dynamic atlas of its own shape.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Rigid motion: pose (q_o, t) moves a Gaussian's mean to R(q_o) mu + t and
composes its rotation as q_o * q (Hamilton product), so its covariance
R S^2 R^T becomes R(q_o) R S^2 R^T R(q_o)^T; the optical depth along any ray
through the moved Gaussian equals the rest-pose one along the ray moved back
(Eqs. 2-3 depend on the ray only through o - mu and d).
Two atlases: optical depth is additive (Eq. 1), so the transmittance of the
union of two occluder sets is the product of their transmittances; each
atlas is sampled at its own texel and shell bracket (Sec. 3.3).
"""
from __future__ import annotations

import numpy as np

from . import attenuate as _attenuate


def _unit(q):
    q = np.asarray(q, dtype=np.float64)
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def hamilton(a, b):
    """Row-wise Hamilton product a * b of (w, x, y, z) quaternions."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    aw, av = a[..., :1], a[..., 1:]
    bw, bv = b[..., :1], b[..., 1:]
    w = aw * bw - np.sum(av * bv, axis=-1, keepdims=True)
    v = aw * bv + bw * av + np.cross(av, bv)
    return np.concatenate([w, v], axis=-1)


def quat_rotate(q, v):
    """Rotate vectors v by unit quaternions q: the vector part of q v q*."""
    q = _unit(q)
    qv = np.concatenate([np.zeros(np.shape(v)[:-1] + (1,)), np.asarray(v, dtype=np.float64)], axis=-1)
    conj = q * np.array([1.0, -1.0, -1.0, -1.0])
    return hamilton(hamilton(q, qv), conj)[..., 1:]


def object_of(seg, n):
    seg = np.asarray(seg, dtype=np.int64)
    return np.repeat(np.arange(seg.size - 1), np.diff(seg))[:n]


def rigid_transform(means, quats, seg, poses):
    """(means', quats') in FP64 for contiguous objects seg and poses (n_obj, 8)."""
    means = np.asarray(means, dtype=np.float64)
    quats = np.asarray(quats, dtype=np.float64)
    poses = np.asarray(poses, dtype=np.float64)
    o = object_of(seg, means.shape[0])
    qo = _unit(poses[o, :4])
    return quat_rotate(qo, means) + poses[o, 4:7], hamilton(qo, quats)


def segment_centroids(means, weights, seg):
    means = np.asarray(means, dtype=np.float64)
    w = np.ones(means.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    out = np.zeros((len(seg) - 1, 3))
    for k in range(len(seg) - 1):
        a, b = seg[k], seg[k + 1]
        sw = w[a:b].sum()
        if sw > 0:
            out[k] = (w[a:b, None] * means[a:b]).sum(0) / sw
    return out


def attenuate_two(atlas, radii, atlas_dyn, radii_dyn, lights, q_means, colors, light_w=None,
                  direct_frac=1.0):
    """(colours (Q,3), T (Q,L)): T_l = T_static,l * T_dyn,l, each sampled on
    its own atlas; c' = c (1 - w_d + w_d sum_l w_l T_l)."""
    _, Ts = _attenuate(atlas, radii, lights, q_means, colors, want_T=True)
    _, Td = _attenuate(atlas_dyn, radii_dyn, lights, q_means, colors, want_T=True)
    T = Ts * Td
    L = T.shape[1]
    w = np.full(L, 1.0 / L) if light_w is None else np.asarray(light_w, dtype=np.float64)
    f = 1.0 - direct_frac + direct_frac * (T @ w)
    return np.asarray(colors, dtype=np.float64) * f[:, None], T
