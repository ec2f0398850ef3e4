"""Pins of the oracle's HDRI probe fit (Sec. 3.4, Eqs. 7-8) and radiance
transfer (Sec. 3.5, Eqs. 9-10) against scipy's spherical harmonics, numpy's
dense solver and the closed-form clamped-cosine convolution."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

from paper_2601_01660_b300 import scenes

LM = [(0, 0), (1, -1), (1, 0), (1, 1), (2, -2), (2, -1), (2, 0), (2, 1), (2, 2)]


def real_sh_scipy(d):
    """Real SH (no Condon-Shortley phase), index l^2+l+m, from scipy's complex Y_l^m."""
    d = np.atleast_2d(d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.zeros((d.shape[0], 9))
    for k, (l, m) in enumerate(LM):
        Y = sph_harm_y(l, abs(m), theta, phi)
        if m == 0:
            out[:, k] = Y.real
        elif m > 0:
            out[:, k] = math.sqrt(2) * (-1) ** m * Y.real
        else:
            out[:, k] = math.sqrt(2) * (-1) ** m * Y.imag
    return out


def test_basis_matches_scipy(orc):
    rng = np.random.default_rng(0)
    d = rng.normal(size=(500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ref = real_sh_scipy(d)
    got = np.array([orc.sh_basis(x) for x in d])
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_basis_orthonormal(orc):
    nt, npph = 200, 400
    th = (np.arange(nt) + 0.5) * math.pi / nt
    ph = (np.arange(npph) + 0.5) * 2 * math.pi / npph
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    w = (np.sin(T) * (math.pi / nt) * (2 * math.pi / npph)).ravel()
    B = np.array([orc.sh_basis(x) for x in d])
    G = B.T @ (B * w[:, None])
    np.testing.assert_allclose(G, np.eye(9), atol=1e-4)


def test_fit_recovers_band_limited_signal(orc):
    D, _, w = scenes.cubemap_samples(16, seed=1)
    rng = np.random.default_rng(2)
    A_true = rng.normal(size=(9, 3))
    Y = real_sh_scipy(D.astype(np.float64)) @ A_true
    sh = orc.sh_fit(D, Y, w, lam=0.0)
    np.testing.assert_allclose(sh.T, A_true, atol=2e-5, rtol=1e-5)


def test_fit_constant_environment(orc):
    D, _, w = scenes.cubemap_samples(16, seed=1)
    Y = np.full((D.shape[0], 3), 0.75, np.float32)
    sh = orc.sh_fit(D, Y, w, lam=0.0)
    np.testing.assert_allclose(sh[:, 0], 0.75 * 2 * math.sqrt(math.pi), rtol=1e-9)
    assert np.max(np.abs(sh[:, 1:])) < 1e-9


@pytest.mark.parametrize("lam", [0.0, 1e-3, 0.5])
def test_fit_solves_ridge_normal_equations(orc, lam):
    """Eq. 7 against numpy's dense solve of the same normal equations, with the
    basis taken from scipy."""
    D, Y, w = scenes.cubemap_samples(24, seed=3)
    B = real_sh_scipy(D.astype(np.float64))
    W = w.astype(np.float64)
    G = B.T @ (B * W[:, None]) + lam * np.eye(9)
    A = np.linalg.solve(G, B.T @ (Y.astype(np.float64) * W[:, None]))
    sh = orc.sh_fit(D, Y, w, lam=lam)
    np.testing.assert_allclose(sh.T, A, rtol=1e-7, atol=1e-10)


def test_transfer_constant_environment(orc):
    ell = np.array([0.3, 1.2, 2.0])
    sh = np.zeros((3, 9))
    sh[:, 0] = ell * 2 * math.sqrt(math.pi)
    rng = np.random.default_rng(4)
    for q in (1.0, 2.0, 7.5):
        for _ in range(5):
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            s = orc.transfer_scale(sh, n, q=q, eps=0.0)
            np.testing.assert_allclose(s, ell, rtol=1e-12)


def test_transfer_lambertian_limit_is_clamped_cosine_convolution(orc):
    """For q = 1 and a fine grid, Eq. 10 tends to E(n)/pi with the clamped-cosine
    kernel coefficients pi, 2pi/3, pi/4 for bands 0, 1, 2 (Ramamoorthi and
    Hanrahan 2001)."""
    rng = np.random.default_rng(5)
    sh = rng.normal(scale=0.2, size=(3, 9))
    sh[:, 0] = 3.0
    Ahat = np.array([math.pi] + [2 * math.pi / 3] * 3 + [math.pi / 4] * 5)
    for _ in range(6):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Yn = real_sh_scipy(n)[0]
        ref = (sh * Ahat) @ Yn / math.pi
        got = orc.transfer_scale(sh, n, q=1.0, t_max=100.0, eps=0.0, n_theta=256, n_phi=512)
        np.testing.assert_allclose(got, ref, rtol=2e-4)


def test_transfer_clip(orc):
    sh = np.zeros((3, 9))
    sh[:, 0] = np.array([-1.0, 5.0, 100.0]) * 2 * math.sqrt(math.pi)
    s = orc.transfer_scale(sh, np.array([0, 0, 1.0]), t_max=10.0)
    assert s[0] == 0.0 and s[1] == pytest.approx(5.0, rel=1e-7) and s[2] == 10.0


def test_normal_is_smallest_axis_away_from_centroid(orc):
    rng = np.random.default_rng(6)
    for _ in range(20):
        q = scenes.random_quats(rng, 1)[0].astype(np.float32)
        s = np.float32(rng.uniform(0.01, 0.1, 3))
        mu = np.float32(rng.normal(size=3))
        cen = np.float32(rng.normal(size=3))
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        axis = R[:, int(np.argmin(s))]
        if axis @ (mu - cen) < 0:
            axis = -axis
        np.testing.assert_allclose(orc.gauss_normal(mu, s, q, cen), axis, atol=1e-6)


def test_relight_is_scaled_colour(orc):
    rng = np.random.default_rng(7)
    sc = scenes.cube_scene(30, seed=8)
    sh = rng.normal(scale=0.3, size=(3, 9))
    sh[:, 0] = 2.0
    cen = sc.means.mean(0)
    out = orc.relight(sh, sc, cen, gamma=0.8)
    for g in range(sc.n):
        n = orc.gauss_normal(sc.means[g], sc.scales[g], sc.quats[g], cen)
        s = orc.transfer_scale(sh, n)
        np.testing.assert_allclose(out[g], np.maximum(0, 0.8 * sc.colors[g].astype(np.float64) * s), rtol=1e-12)


def test_relight_and_attenuation_commute(orc):
    """Relighting (Eq. 10: max(0, gamma c s), s clipped to [0, t_max]) and
    the attenuation (Sec. 3.3: c (1 - w_d + w_d sum_l w_l T_l)) each scale a
    Gaussian's colour by a factor that is non-negative and does not depend on
    the colour, so their order does not change the result.  The batched frame
    relies on this: it relights the avatars from their input colours beside
    the dynamic build and attenuates the relit colours afterwards."""
    rng = np.random.default_rng(11)
    occ = scenes.cube_scene(400, seed=12)
    recv = scenes.cube_scene(300, seed=13)
    lights = np.float32([[0, 0, 0], [0.6, -0.4, 0.8]])
    radii = scenes.radii_linear(0.1, 8, 8)
    atlas = orc.build_atlas(occ, lights, 16, 24, radii)
    sh = rng.normal(scale=0.3, size=(3, 9))
    sh[:, 0] = 2.0
    cen = recv.means.mean(0)
    lw, wd = np.float32([0.7, 0.3]), 0.85
    # attenuate, then relight
    att = orc.attenuate(atlas, radii, lights, recv.means, recv.colors, light_w=lw, direct_frac=wd)
    first_att = orc.relight(sh, scenes.Scene(recv.means, recv.scales, recv.quats, recv.opac, np.float32(att)),
                            cen, gamma=0.8, t_max=1.5)
    # relight, then attenuate
    rel = orc.relight(sh, recv, cen, gamma=0.8, t_max=1.5)
    first_rel = orc.attenuate(atlas, radii, lights, recv.means, np.float32(rel), light_w=lw, direct_frac=wd)
    # the attenuation is not trivial: some receivers are in shadow
    f = att / np.maximum(recv.colors.astype(np.float64), 1e-12)
    assert f.min() < 0.9 and f.max() <= 1.0 + 1e-12
    # equal up to the float32 rounding of the intermediate colours
    np.testing.assert_allclose(first_rel, first_att, rtol=2e-7, atol=1e-12)
