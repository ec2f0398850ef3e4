"""Pins of the cubemap probe render (Sec. 3.4): the face axes against the
cubemap sample geometry, a single splat's centre and neighbour pixels in
closed form (EWA covariance of an isotropic Gaussian), front-to-back
compositing order through opaque layers, the near plane, and every face's
projection against the direction table."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_01660_b300 import scenes


def _scene(mus, s, alphas, cols):
    n = len(mus)
    return scenes.Scene(np.float32(mus), np.float32([[s, s, s]] * n), np.float32([[1, 0, 0, 0]] * n),
                        np.float32(alphas), np.float32(cols))


def test_cube_dirs_match_the_sample_geometry():
    D, _, _ = scenes.cubemap_samples(8, seed=0)
    assert np.abs(oracle.cube_dirs(8) - D).max() < 1e-6
    Dc = oracle.cube_dirs(2)
    F = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    for f in range(6):  # each face's texels lean towards its forward axis
        assert (Dc[4 * f:4 * f + 4] @ F[f] > 0.5).all()


def test_single_splat_centre_and_neighbour():
    face, d, s, a = 32, 2.0, 0.02, 0.7
    D = oracle.cube_dirs(face)
    p = 4 * face * face + 10 * face + 21            # face +z, row 10, column 21
    mu = (d * D[p]).astype(np.float32)
    sc = _scene([mu], s, [a], [[0.2, 0.5, 0.9]])
    nb = p + 1                                      # the next column
    rgb = oracle.render_pixels(sc, [0, 0, 0], face, [p, nb])
    # at the centre: alpha = a (m^2 ~ 0, float rounding of the projection)
    assert np.allclose(rgb[0], a * np.float32([0.2, 0.5, 0.9]), rtol=1e-5)
    # the neighbour: EWA of an isotropic Gaussian, the Jacobian at the mean
    fl = face / 2
    t = mu.astype(np.float64)
    tz, tx, ty = t[2], t[0], -t[1]                  # face +z: U = +x, V = -y
    J = (fl / tz) * np.array([[1, 0, -tx / tz], [0, 1, -ty / tz]])
    S2 = J @ (s * s * np.eye(3)) @ J.T + 0.3 * np.eye(2)
    mx, my = (tx / tz + 1) * fl, (ty / tz + 1) * fl
    dvec = np.array([21 + 1 + 0.5 - mx, 10 + 0.5 - my])
    m2 = dvec @ np.linalg.solve(S2, dvec)
    assert m2 < 9
    assert rgb[1] == pytest.approx(a * math.exp(-0.5 * m2) * np.float32([0.2, 0.5, 0.9]), rel=1e-4)


def test_front_to_back_order_and_stop():
    face = 16
    D = oracle.cube_dirs(face)
    p = 4 * face * face + 7 * face + 8
    d = D[p]
    c1, c2, c3 = [1, 0, 0], [0, 1, 0], [0, 0, 1]
    # listed back to front: the render must sort by depth
    sc = _scene([(3.0 * d).astype(np.float32), (2.0 * d).astype(np.float32)], 0.05, [0.6, 0.5], [c2, c1])
    rgb = oracle.render_pixels(sc, [0, 0, 0], face, [p])[0]
    a1, a2 = 0.5, 0.6  # alpha at the splat centre (m^2 ~ 0)
    assert np.allclose(rgb, [a1, (1 - a1) * a2, 0], atol=2e-5)
    # three opaque layers (alpha capped at 0.99): T = 1, 0.01, 1e-4 in front of them
    sc = _scene([(k * d).astype(np.float32) for k in (2.0, 3.0, 4.0)], 0.05, [1.0, 1.0, 1.0], [c1, c2, c3])
    rgb = oracle.render_pixels(sc, [0, 0, 0], face, [p])[0]
    assert np.allclose(rgb, [0.99, 0.01 * 0.99, 1e-4 * 0.99], rtol=1e-4, atol=1e-12)


def test_near_plane_and_transparent():
    face = 16
    D = oracle.cube_dirs(face)
    p = 2 * face * face + 3 * face + 4
    sc = _scene([(0.01 * D[p]).astype(np.float32), (2 * D[p]).astype(np.float32)], 0.05, [0.9, 0.0],
                [[1, 1, 1], [1, 1, 1]])
    assert np.abs(oracle.render_pixels(sc, [0, 0, 0], face, [p], near=0.05)).max() == 0.0


def test_every_face_projects_along_its_directions():
    face = 8
    D = oracle.cube_dirs(face)
    rng = np.random.default_rng(2)
    for p in rng.choice(D.shape[0], 24, replace=False):
        o = np.float32([0.3, -0.2, 1.0])
        sc = _scene([(o + 2.5 * D[p]).astype(np.float32)], 0.01, [0.8], [[1, 1, 1]])
        img = oracle.render_pixels(sc, o, face, np.arange(D.shape[0]))
        assert int(np.argmax(img[:, 0])) == p and img[p, 0] > 0.7


def _camera(rot_seed, pos, fx, fy, cx, cy):
    from scipy.spatial.transform import Rotation
    R = Rotation.random(random_state=rot_seed).as_matrix()  # rows: image x, image y, forward
    return np.float32(np.concatenate([R.ravel(), pos, [fx, fy, cx, cy]])), R


def test_pinhole_camera_projects_view_points_to_their_pixels():
    W, H = 40, 28
    cam, R = _camera(3, [0.2, -0.1, 0.5], 30.0, 28.0, 20.0, 14.0)
    rng = np.random.default_rng(5)
    for _ in range(12):
        i, j = int(rng.integers(2, H - 2)), int(rng.integers(2, W - 2))
        z = float(rng.uniform(1.0, 3.0))
        x, y = (j + 0.5 - 20.0) * z / 30.0, (i + 0.5 - 14.0) * z / 28.0
        mu = np.float32([0.2, -0.1, 0.5]) + R.T @ np.array([x, y, z])
        sc = _scene([mu.astype(np.float32)], 0.004, [0.8], [[1, 1, 1]])
        img = oracle.render_view_pixels(sc, cam[None], W, H, np.arange(W * H))
        assert int(np.argmax(img[:, 0])) == i * W + j
        assert img[i * W + j, 0] == pytest.approx(0.8, rel=1e-4)


def test_cube_face_is_a_camera():
    sc = scenes.cube_scene(300, seed=6, centre=(0.0, 0.0, 0.0), side=5.0)
    face = 8
    cams = oracle.cube_cams([0.1, 0.2, -0.3], face)
    a = oracle.render_pixels(sc, [0.1, 0.2, -0.3], face, np.arange(6 * face * face))
    b = oracle.render_view_pixels(sc, cams, face, face, np.arange(6 * face * face))
    assert np.array_equal(a, b)
    # the camera rows are the face axes of the direction table
    D = oracle.cube_dirs(face).reshape(6, face, face, 3)
    for f in range(6):
        centre_dir = D[f, face // 2 - 1:face // 2 + 1, face // 2 - 1:face // 2 + 1].mean((0, 1))
        assert np.dot(centre_dir / np.linalg.norm(centre_dir), cams[f, 6:9]) > 0.999
