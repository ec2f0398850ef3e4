"""Pins of the opacity-to-absorption mappings (ablation (B) of Sec. 4): each
mapping's optical depth through the centre of an isotropic Gaussian in
closed form, mappings 3 and 4 equal for 3DGS covariances, and the culling
radius of each mapping bounding the optical depth a missed ray carries."""
import math

import numpy as np
import pytest

from paper_2601_01660_b300 import scenes


def _one(mu, s, alpha, quat=(1, 0, 0, 0)):
    return scenes.Scene(np.float32([mu]), np.float32([s]), np.float32([quat]), np.float32([alpha]),
                        np.float32([[1, 1, 1]]))


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_line_through_isotropic_centre(orc, mode):
    """Along a full line through the centre of an isotropic Gaussian of scale
    s the line integral of exp(-q/2) is s sqrt(2 pi), so tau = beta s sqrt(2 pi):
    kappa tau* s sqrt(2 pi) (1), kappa tau* (2, the calibration of Eq. 5),
    kappa tau* / (2 pi s^2) (3, 4)."""
    for alpha, s, kappa in [(0.3, 0.05, 1.0), (0.9, 0.2, 1.0), (0.5, 0.1, 2.0)]:
        sc = _one([0, 0, 4.0], [s, s, s], alpha)
        ts = -math.log1p(-float(np.float32(alpha)))
        s32 = float(np.float32(s))
        ref = {1: kappa * ts * s32 * math.sqrt(2 * math.pi), 2: kappa * ts,
               3: kappa * ts / (2 * math.pi * s32 * s32), 4: kappa * ts / (2 * math.pi * s32 * s32)}[mode]
        with orc.beta_mode(mode):
            tau = orc.tau_rays(sc, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), [8.0], kappa)[0]
        assert tau == pytest.approx(ref, rel=1e-9)


def test_mappings_3_and_4_agree(orc):
    """sqrt(det Sigma) of Sigma = R diag(s^2) R^T equals s_x s_y s_z."""
    sc = scenes.cube_scene(50, seed=9)
    d = np.array([[0.1, -0.2, 1.0]]) / np.linalg.norm([0.1, -0.2, 1.0])
    for i in range(sc.n):
        one = scenes.subset(sc, [i])
        with orc.beta_mode(3):
            t3 = orc.tau_rays(one, np.zeros((1, 3)), d, [9.0])[0]
        with orc.beta_mode(4):
            t4 = orc.tau_rays(one, np.zeros((1, 3)), d, [9.0])[0]
        assert t3 == pytest.approx(t4, rel=1e-9, abs=1e-300)


def test_mode_is_restored(orc):
    with orc.beta_mode(1):
        with orc.beta_mode(3):
            assert orc.lib().orc_get_beta_mode() == 3
        assert orc.lib().orc_get_beta_mode() == 1
    assert orc.lib().orc_get_beta_mode() == 2


@pytest.mark.parametrize("mode", [1, 3])
def test_cull_radius_bounds_missed_optical_depth(orc, mode):
    """A ray outside the k-ellipsoid of mapping `mode` carries at most eps."""
    rng = np.random.default_rng(6)
    sc = scenes.cube_scene(40, seed=14)
    eps = 1e-7
    checked = 0
    with orc.beta_mode(mode):
        for i in range(sc.n):
            r, g = orc.f32_gauss_cone(sc.means[i], sc.scales[i], sc.opac[i], np.zeros(3), 1.0, eps, 1e9)
            k = math.sqrt(g[6])
            A = orc.precision(sc.scales[i], sc.quats[i])
            Rm = orc.rotation(sc.quats[i])
            one = scenes.subset(sc, [i])
            for _ in range(8):
                z = rng.normal(size=3)
                z /= np.linalg.norm(z)
                p = sc.means[i] + Rm @ (z * 1.02 * k * sc.scales[i])
                d = p / np.linalg.norm(p)
                a, b, c = orc.ray_coeffs(A, d, -sc.means[i].astype(np.float64))
                if c - b * b / a < k * k:
                    continue
                tau = orc.tau_rays(one, np.zeros((1, 3)), d[None], [1e4])[0]
                assert tau <= eps * 1.0001
                checked += 1
    assert checked > 50
