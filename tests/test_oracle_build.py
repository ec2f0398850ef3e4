"""Pins of the oracle's DGSM build (Sec. 3.2, Eqs. 1-5) against things other
than itself: numerical quadrature, an independent rotation library, the
opacity calibration the paper states for Eq. 5, and invariants of Eqs. 2/4."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

from paper_2601_01660_b300 import scenes


def _quad(f, lo, hi):
    val, err = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=400)
    return val


@pytest.mark.parametrize("a,b,c,t", [
    (4.0, -6.0, 10.0, 3.0),        # closest approach inside [0,t]: straddling case
    (2.5, 3.0, 5.0, 2.0),          # closest approach behind the origin: x0 >= 0
    (9.0, -40.0, 180.0, 1.0),      # closest approach beyond t: xt <= 0
    (1e4, -3e4, 9.0001e4, 5.0),    # thin Gaussian crossed at 3 m
    (0.3, -0.1, 0.04, 12.0),       # wide Gaussian around the origin
    (50.0, -300.0, 1800.5, 8.0),
])
def test_eq3_matches_quadrature_of_eq2(orc, a, b, c, t):
    """Eq. 3 equals the integral it closes (Eq. 2) to 1e-10 relative."""
    ref = _quad(lambda s: math.exp(-0.5 * (a * s * s + 2 * b * s + c)), 0.0, t)
    # split the quadrature at the peak so quad sees it
    s_star = -b / a
    if 0 < s_star < t:
        ref = (_quad(lambda s: math.exp(-0.5 * (a * s * s + 2 * b * s + c)), 0.0, s_star) +
               _quad(lambda s: math.exp(-0.5 * (a * s * s + 2 * b * s + c)), s_star, t))
    got = orc.line_integral(a, b, c, t)
    assert got == pytest.approx(ref, rel=1e-10, abs=1e-300)


def test_rotation_matches_scipy(orc):
    rng = np.random.default_rng(11)
    for _ in range(20):
        q = scenes.random_quats(rng, 1)[0].astype(np.float32)
        R_ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: scalar last
        np.testing.assert_allclose(orc.rotation(q), R_ref, atol=1e-6)


def _density(sc, x, betas):
    """Eq. 1 evaluated directly: sigma(x) = sum_i beta_i exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),
    with Sigma = R diag(s^2) R^T from scipy's rotation."""
    acc = 0.0
    for i in range(sc.n):
        q = sc.quats[i].astype(np.float64)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(sc.scales[i].astype(np.float64) ** 2) @ R.T
        dx = x - sc.means[i]
        acc += betas[i] * math.exp(-0.5 * dx @ np.linalg.solve(Sig, dx))
    return acc


def test_tau_matches_quadrature_of_density(orc):
    """tau(d,t) of Eq. 2 equals the quadrature of the Eq. 1 density along the ray."""
    sc = scenes.cube_scene(5, seed=21, centre=(0, 0, 2.0), side=1.0, log_s_mean=math.log(0.2),
                           log_s_std=0.4)
    betas = [orc.beta(sc.scales[i], sc.opac[i], 1.0) for i in range(sc.n)]
    rng = np.random.default_rng(3)
    o = np.array([0.1, -0.05, 0.0])
    for r in range(6):
        target = sc.means[r % sc.n] + rng.normal(0, 0.1, 3)
        d = (target - o) / np.linalg.norm(target - o)
        t = float(np.linalg.norm(target - o)) + rng.uniform(-0.3, 0.6)
        ref = _quad(lambda s: _density(sc, o + s * d, betas), 0.0, t)
        got = orc.tau_rays(sc, o[None], d[None], [t])[0]
        assert got == pytest.approx(ref, rel=1e-8)


def test_isotropic_calibration_T_equals_one_minus_alpha(orc):
    """Eq. 5 is calibrated so that an isotropic Gaussian crossed through its
    centre, far from the light and fully traversed, gives T = (1-alpha)^kappa:
    the optical depth 3DGS alpha compositing implies (Sec. 3.2)."""
    for alpha, s, kappa in [(0.3, 0.05, 1.0), (0.9, 0.2, 1.0), (0.5, 0.01, 2.0), (0.05, 0.5, 0.7)]:
        sc = scenes.Scene(np.float32([[0, 0, 4.0]]), np.float32([[s, s, s]]),
                          np.float32([[1, 0, 0, 0]]), np.float32([alpha]), np.float32([[1, 1, 1]]))
        tau = orc.tau_rays(sc, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), [8.0], kappa)[0]
        a32 = float(np.float32(alpha))  # the opacity as the float32 input holds it
        assert math.exp(-tau) == pytest.approx((1 - a32) ** kappa, rel=1e-7)


def test_isotropic_closed_form_off_axis(orc):
    """For A = I/s^2, Eqs. 3+5 reduce to
    tau = 1/2 kappa tau* exp(-h^2/2s^2) [erf((t-p)/(s sqrt2)) + erf(p/(s sqrt2))],
    p the ray parameter of closest approach, h the miss distance."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        s = float(np.float32(rng.uniform(0.05, 0.5)))
        alpha = float(np.float32(rng.uniform(0.05, 0.95)))
        mu = np.float32(rng.uniform(-1, 1, 3) + [0, 0, 3])
        sc = scenes.Scene(mu[None], np.float32([[s, s, s]]), np.float32([[1, 0, 0, 0]]),
                          np.float32([alpha]), np.float32([[1, 1, 1]]))
        d = rng.normal(size=3) + [0, 0, 3]
        d /= np.linalg.norm(d)
        t = rng.uniform(0.5, 6.0)
        mu64 = mu.astype(np.float64)
        p = d @ mu64
        h = np.linalg.norm(mu64 - p * d)
        ts = -math.log1p(-alpha)
        ref = 0.5 * ts * math.exp(-h * h / (2 * s * s)) * (
            math.erf((t - p) / (s * math.sqrt(2))) + math.erf(p / (s * math.sqrt(2))))
        got = orc.tau_rays(sc, np.zeros((1, 3)), d[None], [t])[0]
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-15)


def test_anisotropic_trace_proxy(orc):
    """Eq. 5 replaces sqrt(a) by the direction-agnostic sqrt(tr(A)/3); along the
    local direction R (1,1,1)/sqrt3, where d^T A d = tr(A)/3 exactly, a full
    crossing through the centre again gives T = 1 - alpha."""
    rng = np.random.default_rng(9)
    for _ in range(8):
        s = np.float32(np.exp(rng.normal(math.log(0.05), 0.5, 3)))
        q = scenes.random_quats(rng, 1)[0].astype(np.float32)
        alpha = float(np.float32(rng.uniform(0.05, 0.95)))
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        d = R @ (np.ones(3) / math.sqrt(3))
        mu = np.float32(d * 4.0)
        sc = scenes.Scene(mu[None], s[None], q[None], np.float32([alpha]), np.float32([[1, 1, 1]]))
        d = mu.astype(np.float64) / np.linalg.norm(mu.astype(np.float64))
        tau = orc.tau_rays(sc, np.zeros((1, 3)), d[None], [8.0])[0]
        assert math.exp(-tau) == pytest.approx(1 - alpha, rel=1e-6)


def test_empty_scene_is_fully_lit(orc):
    sc = scenes.cube_scene(0, seed=0)
    T = orc.build_atlas(sc, [[0, 0, 0]], 8, 8, scenes.radii_linear(0.1, 8, 4))
    assert T.shape == (1, 4, 8, 8)
    assert np.all(T == 1.0)


def test_zero_opacity_contributes_nothing(orc):
    sc = scenes.cube_scene(50, seed=4)
    sc.opac[:] = 0.0
    tau = orc.build_tau(sc, [[0, 0, 0]], 8, 8, scenes.radii_linear(0.1, 8, 4))
    assert np.all(tau == 0.0)


def test_T_bounds_and_monotone_in_radius(orc):
    sc = scenes.cube_scene(300, seed=6)
    T = orc.build_atlas(sc, [[0, 0, 0], [0.5, 0.2, 1.0]], 16, 12, scenes.radii_linear(0.1, 8, 10))
    assert np.all(T > 0) and np.all(T <= 1)
    assert np.all(np.diff(T, axis=1) <= 0)


def test_gaussian_behind_light_is_invisible(orc):
    """A small Gaussian on the far side of the light adds (almost) nothing to
    tau in the opposite hemisphere (Eq. 2 integrates t >= 0 only)."""
    base = scenes.cube_scene(40, seed=8)
    extra = scenes.Scene(np.float32([[0, 0, -2.0]]), np.float32([[0.05, 0.05, 0.05]]),
                         np.float32([[1, 0, 0, 0]]), np.float32([0.9]), np.float32([[1, 1, 1]]))
    radii = scenes.radii_linear(0.1, 8, 6)
    t0 = orc.build_tau(base, [[0, 0, 0]], 16, 16, radii)
    t1 = orc.build_tau(scenes.concat(base, extra), [[0, 0, 0]], 16, 16, radii)
    up = np.zeros((16, 16), bool)
    for i in range(16):
        for j in range(16):
            up[i, j] = orc.texel_dir(i, j, 16, 16)[2] > 0
    assert np.abs(t1 - t0)[:, :, up].max() < 1e-300
