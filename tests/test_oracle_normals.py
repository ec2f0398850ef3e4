"""Pins of the local-PCA pseudo-normals (Sec. 4): Gaussians on a plane get
the plane's normal, the normal minimises the weighted second moment over a
dense sample of the sphere, a symmetric configuration in which the distance
weight (not the spread) picks the axis, zero-opacity and out-of-radius
Gaussians change nothing, the smallest-axis fallback against scipy's
rotations, the orientation rule, and rigid-motion equivariance."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import normals as onorm


def _cloud_on_plane(rng, n, nu, origin, half=0.3):
    nu = np.asarray(nu, float) / np.linalg.norm(nu)
    a = np.cross(nu, [1.0, 0, 0] if abs(nu[0]) < 0.9 else [0, 1.0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(nu, a)
    uv = rng.uniform(-half, half, (n, 2))
    return np.asarray(origin, float) + uv[:, :1] * a + uv[:, 1:] * b, nu


def _iso(n):
    return np.tile([1.0, 0, 0, 0], (n, 1)), np.full((n, 3), 0.01)


def test_plane_gives_its_normal():
    rng = np.random.default_rng(0)
    x, nu = _cloud_on_plane(rng, 400, [0.3, -0.2, 1.0], [0.5, 0.2, 1.0])
    q, s = _iso(400)
    op = rng.uniform(0.1, 1.0, 400)
    centroid = np.array([0.5, 0.2, 1.0]) - 2.0 * nu       # below the plane
    nrm, lam, fb = onorm.pca_normals(x, op, q, s, 0.12, centroid, want_info=True)
    assert not fb.any()
    assert np.abs(nrm - nu).max() < 1e-10                  # all turned away from the centroid
    assert np.abs(lam[:, 0]).max() < 1e-14 and lam[:, 1].min() > 1e-5


def test_normal_minimises_the_weighted_second_moment():
    rng = np.random.default_rng(1)
    x = rng.normal(0, 0.05, (60, 3)) * [1.0, 0.6, 0.25]
    op = rng.uniform(0.05, 1.0, 60)
    q, s = _iso(60)
    nrm = onorm.pca_normals(x, op, q, s, 0.2, np.zeros(3))
    # dense sphere sample (Fibonacci lattice)
    k = np.arange(20000) + 0.5
    phi = np.arccos(1 - 2 * k / k.size)
    th = np.pi * (1 + 5 ** 0.5) * k
    S = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    for i in range(0, 60, 7):
        d = x - x[i]
        d2 = (d * d).sum(1)
        w = np.where(d2 <= 0.04, op * (1 - d2 / 0.04) ** 2, 0.0)
        m = (w[:, None] * d).sum(0) / w.sum()
        e = d - m

        def moment(v):
            return float((w * (e @ v) ** 2).sum() / w.sum())
        best = min(moment(v) for v in S)
        assert moment(nrm[i]) <= best * (1 + 1e-9)
        assert abs(np.linalg.norm(nrm[i]) - 1) < 1e-12


def test_distance_weight_picks_the_axis():
    """Pairs at +-0.9 r along x, +-0.5 r along y, +-0.3 r along z, equal
    opacity: the weighted spreads are 2 (1-0.81)^2 0.81, 2 (1-0.25)^2 0.25 and
    2 (1-0.09)^2 0.09 r^2 (over W), smallest along x, although x reaches
    farthest and an unweighted PCA would pick z."""
    r = 0.2
    x = np.zeros((7, 3))
    for k, (ax, f) in enumerate([(0, 0.9), (1, 0.5), (2, 0.3)]):
        x[1 + 2 * k, ax] = f * r
        x[2 + 2 * k, ax] = -f * r
    q, s = _iso(7)
    nrm, lam, _ = onorm.pca_normals(x, np.full(7, 0.5), q, s, r, [-1.0, -1.0, -1.0], want_info=True)
    assert np.allclose(nrm[0], [1, 0, 0], atol=1e-12)
    W = 0.5 * (1 + 2 * (0.19 ** 2 + 0.75 ** 2 + 0.91 ** 2))
    ref = 0.5 * 2 * np.array([0.19 ** 2 * 0.81, 0.75 ** 2 * 0.25, 0.91 ** 2 * 0.09]) * r * r / W
    assert np.allclose(lam[0], np.sort(ref), rtol=1e-12)


def test_transparent_and_far_gaussians_change_nothing():
    rng = np.random.default_rng(2)
    x, nu = _cloud_on_plane(rng, 200, [0, 0, 1.0], [0, 0, 0])
    q, s = _iso(203)
    op = rng.uniform(0.2, 1.0, 200)
    extra = np.array([[0.0, 0.0, 0.05], [0.01, 0.0, -0.04], [0.0, 0.0, 0.2]])  # two transparent, one far
    x2 = np.concatenate([x, extra])
    op2 = np.concatenate([op, [0.0, 0.0, 1.0]])
    a = onorm.pca_normals(x, op, q[:200], s[:200], 0.1, [0, 0, -1.0])
    b = onorm.pca_normals(x2, op2, q, s, 0.1, [0, 0, -1.0])
    near_far = np.linalg.norm(x - extra[2], axis=1) > 0.1
    assert np.abs(a[near_far] - b[:200][near_far]).max() < 1e-12


def test_sparse_neighbourhood_falls_back_to_the_smallest_axis():
    rng = np.random.default_rng(3)
    x = rng.uniform(-5, 5, (20, 3))                          # ~3 m apart: no neighbours
    quats = rng.normal(size=(20, 4))
    scales = np.exp(rng.normal(-3, 0.5, (20, 3)))
    c = np.array([0.1, 0.2, 0.3])
    nrm, _, fb = onorm.pca_normals(x, np.full(20, 0.8), quats, scales, 0.05, c, want_info=True)
    assert fb.all()
    Rm = Rotation.from_quat(quats[:, [1, 2, 3, 0]]).as_matrix()   # scipy takes (x, y, z, w)
    for i in range(20):
        ax = Rm[i][:, np.argmin(scales[i])]
        ax = ax if np.dot(ax, x[i] - c) >= 0 else -ax
        assert np.allclose(nrm[i], ax, atol=1e-12)


def test_orientation_and_rigid_motion():
    rng = np.random.default_rng(4)
    u = rng.normal(size=(2000, 3))
    x = 0.5 * u / np.linalg.norm(u, axis=1, keepdims=True)   # a sphere of radius 0.5
    q, s = _iso(2000)
    op = rng.uniform(0.3, 1.0, 2000)
    nrm = onorm.pca_normals(x, op, q, s, 0.15, np.zeros(3))
    radial = x / 0.5
    cos = np.einsum("nc,nc->n", nrm, radial)
    assert (cos > 0.9).all() and np.median(cos) > 0.995      # outward, close to radial
    R = Rotation.random(random_state=5).as_matrix()
    t = np.array([1.0, -2.0, 0.5])
    moved = onorm.pca_normals(x @ R.T + t, op, q, s, 0.15, t)
    assert np.abs(moved - nrm @ R.T).max() < 1e-9


def test_coincident_neighbourhood_falls_back_and_bad_radius_is_refused():
    """Neighbours that all coincide leave C = 0 (no direction to pick): the
    smallest axis is taken, as for a sparse neighbourhood."""
    q, s = _iso(3)
    s[:, 2] = 0.001
    x = np.tile([0.0, 0.0, 1.0], (3, 1))
    nrm, _, fb = onorm.pca_normals(x, np.ones(3), q, s, 0.1, np.zeros(3), want_info=True)
    assert fb.all() and np.allclose(nrm, [[0, 0, 1.0]] * 3)
    for r in (0.0, -1.0, float("nan")):
        with pytest.raises(ValueError):
            onorm.pca_normals(x, np.ones(3), q, s, r, np.zeros(3))
