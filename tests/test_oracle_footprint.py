"""Pins of the footprint-sampling oracle (Sec. 3.3 last paragraph, ablation (A)
of Sec. 4): the Philox4x64-10 generator against numpy's independent
implementation, the normal numbers against the standard normal law, the
stencil weights, and the sample points against an independent rotation
(scipy) and the centre lookup."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle
from paper_2601_01660_b300 import scenes


@pytest.mark.parametrize("counter,key", [([1, 0, 0, 0], [0, 0]), ([5, 0, 0, 0], [7, 9]),
                                         ([123456789, 3, 0, 0], [2**64 - 1, 1]),
                                         ([2**63, 2**40, 17, 99], [314159, 271828])])
def test_philox_matches_numpy(counter, key):
    # numpy's Philox bit generator advances its counter by one before each
    # block, so it is started one step behind (all counters here have c0 >= 1)
    prev = np.array(counter, dtype=np.uint64)
    prev[0] -= np.uint64(1)
    bg = np.random.Philox(counter=prev, key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4).astype(np.uint64)
    assert np.array_equal(oracle.philox4x64(counter, key), ref)


def test_fp_normals_are_standard_normal():
    z = np.array([oracle.fp_normal(11, q, j) for q in range(1500) for j in range(24)])
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # cos / sin halves of one Box-Muller pair are uncorrelated
    zc, zs = z[0::2], z[1::2]
    assert abs(np.corrcoef(zc, zs)[0, 1]) < 0.03
    # different receivers and seeds draw different numbers
    assert oracle.fp_normal(11, 0, 0) != oracle.fp_normal(11, 1, 0)
    assert oracle.fp_normal(11, 0, 0) != oracle.fp_normal(12, 0, 0)


def test_mc_offsets_follow_the_generator_layout():
    z, w = oracle.fp_offsets("mc", 5, seed=3, q=42)
    assert z.shape == (5, 3) and np.allclose(w, 0.2)
    for i in range(5):
        for c in range(3):
            assert z[i, c] == oracle.fp_normal(3, 42, 3 * i + c)


def test_stencil_weights():
    z, w = oracle.fp_offsets("stencil7")
    assert z.shape == (7, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    ker = np.exp(-0.5 * (z ** 2).sum(1))
    assert np.allclose(w, ker / ker.sum(), rtol=1e-14)
    assert np.allclose(z.sum(0), 0.0)          # symmetric about the centre
    assert np.allclose(np.abs(z).sum(0), 2.0)  # +- one standard deviation per axis


def _cube_atlas(seed=0, n=300, H=16, W=24, K=8):
    sc = scenes.cube_scene(n, seed=seed)
    lights = np.float32([[0, 0, 0], [0.4, -0.3, 0.8]])
    radii = scenes.radii_linear(0.1, 8, K)
    return sc, lights, radii, oracle.build_atlas(sc, lights, H, W, radii)


def test_footprint_points_against_independent_rotation():
    sc, lights, radii, atlas = _cube_atlas()
    q = scenes.cube_scene(40, seed=1)
    for mode, n in (("stencil7", 7), ("mc", 6)):
        _, T = oracle.attenuate_footprint(atlas, radii, lights, q.means, q.quats, q.scales, q.colors,
                                          mode=mode, n_samples=n, seed=5, want_T=True)
        for r in range(q.n):
            z, w = oracle.fp_offsets(mode, n, seed=5, q=r)
            qw, qx, qy, qz = q.quats[r].astype(np.float64)
            Rm = Rotation.from_quat([qx, qy, qz, qw]).as_matrix()  # scipy: scalar last
            pts = q.means[r].astype(np.float64) + (z * q.scales[r].astype(np.float64)) @ Rm.T
            for l in range(lights.shape[0]):
                ref = sum(wi * oracle.sample_T(atlas[l], radii, lights[l].astype(np.float64), p)
                          for wi, p in zip(w, pts))
                assert abs(T[r, l] - ref) < 1e-13


def test_footprint_reduces_to_centre_sample():
    sc, lights, radii, atlas = _cube_atlas(seed=2)
    q = scenes.cube_scene(200, seed=3)
    c_ref, T_ref = oracle.attenuate(atlas, radii, lights, q.means, q.colors, want_T=True)
    c0, T0 = oracle.attenuate_footprint(atlas, radii, lights, q.means, q.quats, q.scales, q.colors,
                                        mode="centre", want_T=True)
    assert np.array_equal(T0, T_ref) and np.array_equal(c0, c_ref)
    tiny = np.full_like(q.scales, 1e-9)
    for mode in ("stencil7", "mc"):
        _, T = oracle.attenuate_footprint(atlas, radii, lights, q.means, q.quats, tiny, q.colors,
                                          mode=mode, want_T=True)
        assert np.abs(T - T_ref).max() < 1e-6


def test_footprint_of_a_constant_field_and_direct_term():
    sc, lights, radii, atlas = _cube_atlas(seed=4)
    atlas[:] = 0.37
    q = scenes.cube_scene(100, seed=5)
    lw = np.float32([0.25, 0.75])
    c, T = oracle.attenuate_footprint(atlas, radii, lights, q.means, q.quats, q.scales, q.colors,
                                      mode="mc", n_samples=9, light_w=lw, direct_frac=0.6,
                                      want_T=True)
    assert np.allclose(T, 0.37, atol=1e-14)
    f = 1 - 0.6 + 0.6 * 0.37
    assert np.allclose(c, q.colors.astype(np.float64) * f, rtol=1e-13)


def test_footprint_smooths_a_shadow_edge():
    # a receiver straddling the edge of an occluder's shadow gets a footprint
    # transmittance between the fully lit and fully shadowed centre values
    H = W = 32
    K = 8
    radii = scenes.radii_linear(0.5, 4.0, K)
    lights = np.float32([[0, 0, 0]])
    atlas = np.ones((1, K, H, W))
    atlas[0, :, :, : W // 2] = 0.2  # shadow over half of the directions
    mu = np.float32([[0.0, 0.0, 2.0]])  # on the edge direction u = 0
    qs = np.float32([[1, 0, 0, 0]])
    col = np.float32([[1, 1, 1]])
    _, Tc = oracle.attenuate(atlas, radii, lights, mu, col, want_T=True)
    _, Tf = oracle.attenuate_footprint(atlas, radii, lights, mu, qs, np.float32([[0.3, 0.3, 0.3]]),
                                       col, mode="stencil7", want_T=True)
    assert 0.2 < Tf[0, 0] < 1.0
    assert math.isclose(Tf[0, 0], 0.6, abs_tol=0.05)  # symmetric stencil across the edge
    assert 0.2 <= Tc[0, 0] <= 1.0
