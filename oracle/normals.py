"""FP64 oracle of the Gaussians' pseudo-normals by local PCA (Sec. 4,
lighting consistency: a unit pseudo-normal per Gaussian from an alpha- and
distance-weighted PCA of the nearby Gaussian centres, or the smallest
ellipsoid axis).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Parity unpinned by the
paper itself (it prints no normals); the pins are geometric: planes,
weighted-moment minimisation by brute force over the sphere, a symmetric
configuration whose answer the distance weight decides, and the fallback.

Definition (the paper names the weighting, not its form; the reading here):
for Gaussian i with centre x_i, its neighbourhood is every Gaussian j
(itself included) with |x_j - x_i|^2 <= r^2, weighted
    w_j = alpha_j (1 - |x_j - x_i|^2 / r^2)^2,
which vanishes continuously at the neighbourhood's edge.  With d_j = x_j - x_i,
W = sum w_j, m = sum w_j d_j / W, the weighted covariance is
    C = sum w_j (d_j - m)(d_j - m)^T / W,
and the pseudo-normal is the unit eigenvector of C's smallest eigenvalue.
When fewer than three neighbours carry weight, or C = 0 (the weighted
neighbours coincide), the normal is the Gaussian's smallest-scale axis (first
on ties).  The radius must be positive.  Either normal is turned to point away
from a reference point (the centroid the relight uses): flipped when
n . (x_i - centroid) < 0.
"""
from __future__ import annotations

import numpy as np


def _smallest_axis(quat, scale):
    q = np.asarray(quat, dtype=np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    # rotation of a unit quaternion (w, x, y, z), columns are the local axes
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    s = np.asarray(scale, dtype=np.float64)
    k = 0
    if s[1] < s[k]:
        k = 1
    if s[2] < s[k]:
        k = 2
    return R[:, k]


def weighted_moments(means, opac, i, radius):
    """(W, m, C, count) of Gaussian i's neighbourhood, FP64."""
    x = np.asarray(means, dtype=np.float64)
    a = np.asarray(opac, dtype=np.float64)
    d = x - x[i]
    d2 = np.einsum("nc,nc->n", d, d)
    r2 = float(radius) ** 2
    near = d2 <= r2
    w = np.where(near, a * (1.0 - d2 / r2) ** 2, 0.0)
    W = w.sum()
    cnt = int(np.count_nonzero(w > 0))
    if W <= 0:
        return 0.0, np.zeros(3), np.zeros((3, 3)), cnt
    m = (w[:, None] * d).sum(0) / W
    e = d - m
    C = np.einsum("n,ni,nj->ij", w, e, e) / W
    return W, m, C, cnt


def pca_normals(means, opac, quats, scales, radius, centroid, want_info=False, idx=None):
    """Pseudo-normals (n, 3) FP64; with want_info also per Gaussian the
    eigenvalues of C in ascending order (n, 3) and whether the smallest-axis
    fallback was taken (n,).  idx: only these Gaussians (rows in idx order),
    their neighbourhoods still taken from all of them."""
    if not float(radius) > 0:
        raise ValueError("radius must be > 0")
    x = np.asarray(means, dtype=np.float64)
    rows = np.arange(x.shape[0]) if idx is None else np.asarray(idx)
    n = rows.shape[0]
    c = np.asarray(centroid, dtype=np.float64)
    out = np.zeros((n, 3))
    lam = np.zeros((n, 3))
    fb = np.zeros(n, dtype=bool)
    for r_, i in enumerate(rows):
        W, m, C, cnt = weighted_moments(x, opac, i, radius)
        if cnt < 3 or not np.trace(C) > 0:
            v = _smallest_axis(quats[i], scales[i])
            fb[r_] = True
        else:
            ev, V = np.linalg.eigh(C)   # ascending eigenvalues
            lam[r_] = ev
            v = V[:, 0]
        v = v / np.linalg.norm(v)
        if np.dot(v, x[i] - c) < 0:
            v = -v
        out[r_] = v
    return (out, lam, fb) if want_info else out
