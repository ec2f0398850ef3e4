"""Pins of the FP64 oracle of rigid object motion, per-object centroids and
two-atlas attenuation (oracle/motion.py), each against something other than
its own formula: the C oracle's rotation matrices, the ray invariance of the
line integral (Eqs. 2-3), and the C oracle's same-geometry attenuation."""
import math

import numpy as np

from oracle import motion
from paper_2601_01660_b300 import scenes


def _poses(rng, n):
    q = rng.standard_normal((n, 4))
    t = rng.uniform(-2, 2, (n, 3))
    return np.concatenate([q, t, np.zeros((n, 1))], axis=1)


def test_hamilton_product_composes_rotations(orc):
    rng = np.random.default_rng(1)
    a = rng.standard_normal((50, 4))
    b = rng.standard_normal((50, 4))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    ab = motion.hamilton(a, b)
    for k in range(50):
        np.testing.assert_allclose(orc.rotation(ab[k]), orc.rotation(a[k]) @ orc.rotation(b[k]),
                                   atol=1e-6)
    # quaternion rotation of a vector is the matrix of the C oracle
    v = rng.standard_normal((50, 3))
    rv = motion.quat_rotate(a, v)
    for k in range(50):
        np.testing.assert_allclose(rv[k], orc.rotation(a[k]) @ v[k], atol=1e-6)
    # the identity and a quarter turn about z
    np.testing.assert_allclose(motion.quat_rotate([1, 0, 0, 0], [1.0, 2.0, 3.0]), [1, 2, 3])
    h = math.sqrt(0.5)
    np.testing.assert_allclose(motion.quat_rotate([h, 0, 0, h], [1.0, 0.0, 0.0]), [0, 1, 0], atol=1e-15)


def test_rigid_transform_moves_the_covariance(orc):
    rng = np.random.default_rng(2)
    sc = scenes.cube_scene(40, seed=3)
    seg = [0, 15, 15, 40]
    poses = _poses(rng, 3)
    m2, q2 = motion.rigid_transform(sc.means, sc.quats, seg, poses)
    obj = motion.object_of(seg, sc.n)
    for g in range(sc.n):
        Ro = orc.rotation(poses[obj[g], :4] / np.linalg.norm(poses[obj[g], :4]))
        A = orc.precision(sc.scales[g], sc.quats[g])
        A2 = orc.precision(sc.scales[g], q2[g] / np.linalg.norm(q2[g]))
        np.testing.assert_allclose(A2, Ro @ A @ Ro.T, rtol=1e-5, atol=1e-3 * np.abs(A).max())
        np.testing.assert_allclose(m2[g], Ro @ sc.means[g] + poses[obj[g], 4:7], atol=1e-6)


def test_optical_depth_is_invariant_under_motion(orc):
    """tau through the moved Gaussians from o along d equals tau through the
    rest pose along the ray moved back: R^T (o - t), R^T d."""
    rng = np.random.default_rng(4)
    sc = scenes.cube_scene(60, seed=5, log_s_mean=math.log(0.2))
    pose = _poses(rng, 1)
    m2, q2 = motion.rigid_transform(sc.means, sc.quats, [0, sc.n], pose)
    moved = scenes.Scene(np.float32(m2), sc.scales, np.float32(q2 / np.linalg.norm(q2, axis=1, keepdims=True)),
                         sc.opac, sc.colors)
    R = orc.rotation(pose[0, :4] / np.linalg.norm(pose[0, :4]))
    t = pose[0, 4:7]
    o = rng.uniform(-1, 1, (200, 3)) + (R @ np.array([0, 0, 3.0]) + t)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ts = rng.uniform(0.5, 8, 200)
    tau_moved = orc.tau_rays(moved, o, d, ts)
    tau_rest = orc.tau_rays(sc, (o - t) @ R, d @ R, ts)
    assert tau_moved.max() > 0.1
    np.testing.assert_allclose(tau_moved, tau_rest, rtol=2e-4, atol=1e-7)


def test_segment_centroids_follow_the_motion():
    rng = np.random.default_rng(6)
    sc = scenes.cube_scene(300, seed=7)
    seg = [0, 100, 250, 300]
    c0 = motion.segment_centroids(sc.means, sc.opac, seg)
    poses = _poses(rng, 3)
    m2, _ = motion.rigid_transform(sc.means, sc.quats, seg, poses)
    c1 = motion.segment_centroids(m2, sc.opac, seg)
    for k in range(3):
        np.testing.assert_allclose(c1[k], motion.quat_rotate(poses[k, :4], c0[k]) + poses[k, 4:7],
                                   atol=1e-12)
    # equal weights on two points: the midpoint; an empty object: zero
    c = motion.segment_centroids(np.array([[0, 0, 0], [2, 4, 6.0]]), None, [0, 2, 2])
    np.testing.assert_allclose(c, [[1, 2, 3], [0, 0, 0]])


def test_two_atlas_attenuation_reduces_to_the_c_oracle(orc):
    rng = np.random.default_rng(8)
    L, K, H, W = 2, 6, 20, 24
    radii = scenes.radii_geometric(0.1, 8, K)
    atlas = np.sort(rng.random((L, K, H, W)), axis=1)[:, ::-1].copy()
    dyn = np.sort(rng.random((L, K, H, W)), axis=1)[:, ::-1].copy()
    lights = np.float32([[0, 0, 0], [1, 0.5, -0.5]])
    q = np.float32(rng.uniform(-6, 6, (3000, 3)))
    c = np.float32(rng.random((3000, 3)))
    lw = np.float32([0.7, 0.3])
    out, T = motion.attenuate_two(atlas, radii, dyn, radii, lights, q, c, light_w=lw, direct_frac=0.6)
    ref, Tref = orc.attenuate(atlas, radii, lights, q, c, atlas_dyn=dyn, light_w=lw, direct_frac=0.6,
                              want_T=True)
    np.testing.assert_allclose(T, Tref, atol=1e-12)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    # a dynamic atlas of ones at another resolution changes nothing
    ones = np.ones((L, 4, 8, 12))
    out1, T1 = motion.attenuate_two(atlas, radii, ones, scenes.radii_linear(0.2, 5, 4), lights, q, c)
    ref1, Tref1 = orc.attenuate(atlas, radii, lights, q, c, want_T=True)
    np.testing.assert_allclose(T1, Tref1, atol=1e-12)
    np.testing.assert_allclose(out1, ref1, atol=1e-12)
