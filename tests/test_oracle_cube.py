"""Pins of the cube-map atlas (the parameterisation ablation (C) of Sec. 4
compares with the octahedral map of Sec. 3.2): six F x F faces stacked in
rows (H = 6F, W = F).  The texel directions against the probe's cube-map
table, encode and decode against known directions and each other, the FP32
index specification against the FP64 encode, lookups that stay on their
face, the build's calibration along a texel ray, the binning's tile cones,
planes and lists against brute force, and the receiver region."""
import math

import numpy as np
import pytest

from paper_2601_01660_b300 import scenes

from test_oracle_octa_bin import IDX, _brute_lists, _scene_with_flat_and_tiny


def test_texel_dirs_are_the_probe_cube_directions(orc):
    F = 8
    ref = orc.cube_dirs(F)   # pinned against the cube-map sample geometry
    with orc.atlas_map(1):
        got = np.array([orc.texel_dir(i, j, 6 * F, F) for i in range(6 * F) for j in range(F)])
    assert np.abs(got - ref).max() < 1e-12
    assert orc.lib().orc_get_atlas_map() == 0


def test_encode_known_directions_and_ties(orc):
    n = math.sqrt(1 + 0.25 + 0.0625)
    cases = [((1, 0, 0), (0, 0.0, 0.0)), ((0, 0, -1), (5, 0.0, 0.0)), ((0, -2, 0), (3, 0.0, 0.0)),
             ((1, 0.5, -0.25), (0, 0.25, -0.5)),      # face +x: u = -z / x, v = -y / x
             ((0.5, 0.25, 1), (4, 0.5, -0.25)),       # face +z: u = x / z, v = -y / z
             ((1, 1, 0), (0, 0.0, -1.0)),             # |x| = |y|: x wins
             ((-1, 1, 0), (1, 0.0, -1.0)),
             ((0, 1, -1), (2, 0.0, -1.0))]            # |y| = |z|: y wins
    for d, (f, u, v) in cases:
        got = orc.cube_encode(np.array(d, float) / (n if d == (1, 0.5, -0.25) else 1.0))
        assert got[0] == f and got[1] == pytest.approx(u, abs=1e-15) and got[2] == pytest.approx(v, abs=1e-15)


def test_encode_decode_inverse(orc):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        f, u, v = orc.cube_encode(d)
        assert -1 <= u <= 1 and -1 <= v <= 1
        assert np.argmax(np.abs(d)) == f // 2 and (d[f // 2] >= 0) == (f % 2 == 0)
        assert np.abs(orc.cube_decode(f, u, v) - d).max() < 1e-14


@pytest.mark.parametrize("F", [8, 40, 128])
def test_f32_round_trip_every_texel(orc, F):
    """encode(decode(texel centre)) lands in the same texel under the FP32 spec."""
    H = 6 * F
    with orc.atlas_map(1):
        dirs = np.array([orc.texel_dir(i, j, H, F) for i in range(H) for j in range(F)])
        ints, fl = orc.f32_sample_index((dirs * 3.0).astype(np.float32), np.zeros(3), H, F,
                                        scenes.radii_linear(0.1, 8, 4))
    ii, jj = np.meshgrid(np.arange(H), np.arange(F), indexing="ij")
    assert np.array_equal(ints[:, 0], ii.ravel())
    assert np.array_equal(ints[:, 1], jj.ravel())
    for base, cell, fr in ((ints[:, 2], ii.ravel(), fl[:, 0]), (ints[:, 3], jj.ravel(), fl[:, 1])):
        assert np.all(((base == cell) & (fr < 1e-3)) | ((base == cell - 1) & (fr > 1 - 1e-3)))


def test_f32_index_agrees_with_fp64_encode(orc):
    rng = np.random.default_rng(1)
    F = 64
    radii = scenes.radii_geometric(0.05, 12, 20)
    o = np.float32([0.3, -0.2, 1.0])
    pts = np.float32(rng.uniform(-6, 6, (3000, 3)))
    with orc.atlas_map(1):
        ints, fl = orc.f32_sample_index(pts, o, 6 * F, F, radii)
    for p, iv, fv in zip(pts, ints, fl):
        v = p.astype(np.float64) - o
        t = np.linalg.norm(v)
        f, u, vv = orc.cube_encode(v / t)
        gx = (u + 1) / 2 * F - 0.5
        gy = (vv + 1) / 2 * F - 0.5
        assert iv[0] // F == f
        assert iv[3] + fv[1] == pytest.approx(gx, abs=2e-4)
        assert iv[2] - f * F + fv[0] == pytest.approx(gy, abs=2e-4)
        k = int(np.sum(radii.astype(np.float64) <= t)) - 1
        assert abs(iv[4] - k) <= 1 and fv[2] == pytest.approx(t, rel=1e-6)


def test_sample_at_voxel_centre_returns_voxel(orc):
    rng = np.random.default_rng(7)
    K, F = 5, 10
    radii = scenes.radii_geometric(0.2, 9.0, K)
    atlas = rng.random((K, 6 * F, F))
    o = np.array([0.5, -0.25, 1.0])
    with orc.atlas_map(1):
        for _ in range(80):
            k, i, j = rng.integers(K), rng.integers(6 * F), rng.integers(F)
            x = o + orc.texel_dir(i, j, 6 * F, F) * float(radii[k])
            assert orc.sample_T(atlas, radii, o, x) == pytest.approx(atlas[k, i, j], abs=1e-9)


def test_sample_is_trilinear_within_a_face_and_stays_on_it(orc):
    """An atlas linear in (column, row within the face, r) plus 100 x face is
    reproduced exactly between texel centres; near the face edge the clamp
    keeps the taps on the face (the 100 x face term never mixes)."""
    K, F = 6, 16
    radii = scenes.radii_linear(0.5, 5.5, K)
    kk, ii, jj = np.meshgrid(np.arange(K), np.arange(6 * F), np.arange(F), indexing="ij")
    atlas = 0.01 * jj + 0.02 * (ii % F) + 100.0 * (ii // F) + 0.1 * radii.astype(np.float64)[kk]
    rng = np.random.default_rng(8)
    with orc.atlas_map(1):
        for _ in range(300):
            f = int(rng.integers(6))
            u, v = rng.uniform(-1, 1, 2)
            d = orc.cube_decode(f, u, v)
            t = rng.uniform(0.6, 5.4)
            gx = np.clip((u + 1) / 2 * F - 0.5, 0, F - 1)
            gy = np.clip((v + 1) / 2 * F - 0.5, 0, F - 1)
            ref = 0.01 * gx + 0.02 * gy + 100.0 * f + 0.1 * t
            assert orc.sample_T(atlas, radii, np.zeros(3), d * t) == pytest.approx(ref, abs=1e-9)


def test_build_calibration_along_a_texel_ray(orc):
    """An isotropic Gaussian centred on the ray of texel (i, j), far inside the
    last shell: that texel gives T = 1 - alpha (Eq. 5's calibration), and the
    texel on the opposite face sees nothing."""
    F = 8
    radii = np.float32([0.5, 9.0])
    with orc.atlas_map(1):
        for (i, j) in [(3, 4), (2 * F + 1, 6), (5 * F + 7, 0)]:
            d = orc.texel_dir(i, j, 6 * F, F)
            sc = scenes.Scene(np.float32([4.0 * d]), np.float32([[0.05] * 3]), np.float32([[1, 0, 0, 0]]),
                              np.float32([0.6]), np.float32([[1, 1, 1]]))
            T = orc.build_atlas(sc, np.zeros((1, 3), np.float32), 6 * F, F, radii)[0]
            assert T[1, i, j] == pytest.approx(1 - float(np.float32(0.6)), rel=1e-5)
            assert T[0, i, j] == 1.0
            f = i // F
            opp = (f ^ 1) * F + (i - f * F)
            assert T[1, opp, j] == 1.0


@pytest.mark.parametrize("F,tile", [(16, 8), (20, 8), (32, 16), (12, 4), (208, 64), (40, 64)])
def test_tile_cones_contain_their_texels(orc, F, tile):
    """Every rectangle's cone holds its texel rays, also for rectangles across
    two faces (super-tiles of 64 texels on faces of 208 or 40): their cone
    covers both parts (the whole sphere when the two faces are opposite)."""
    H = 6 * F
    across = 0
    with orc.atlas_map(1):
        for i0 in range(0, H, tile):
            for j0 in range(0, F, tile):
                i1, j1 = min(i0 + tile, H), min(j0 + tile, F)
                cone = orc.f32_rect_cone(i0, i1, j0, j1, H, F)
                two = (i1 - 1) // F == i0 // F + 1
                across += two
                if cone[5]:
                    continue
                c = cone[:3].astype(np.float64)
                for i in range(i0, i1, max(1, tile // 16)):
                    for j in range(j0, j1, max(1, tile // 16)):
                        assert orc.texel_dir(i, j, H, F) @ c >= cone[3] - 1e-6
                for i in (i0, i1 - 1):           # the corners always
                    for j in (j0, j1 - 1):
                        assert orc.texel_dir(i, j, H, F) @ c >= cone[3] - 1e-6
    assert across > 0 or F % tile == 0


def test_rect_planes_bound_their_texels(orc):
    F = 24
    H = 6 * F
    with orc.atlas_map(1):
        for (i0, i1, j0, j1) in [(0, 8, 0, 8), (16, 24, 8, 16), (40, 48, 16, 24), (3 * F + 8, 3 * F + 16, 0, 8),
                                 (5 * F + 16, 5 * F + 24, 16, 24), (3, 11, 5, 13)]:
            pl = orc.f32_rect_planes(i0, i1, j0, j1, 4, H, F)
            assert pl[15] == 1
            for i in range(i0, i1):
                for j in range(j0, j1):
                    d = orc.texel_dir(i, j, H, F)
                    for q in range(4):
                        assert pl[3 * q: 3 * q + 3] @ d >= -1e-6
                    side = pl[12:15] @ d
                    assert (side >= -1e-6) if i < i0 + 4 else (side <= 1e-6)
        # a tile across two faces and a one-row tile have no planes
        assert orc.f32_rect_planes(F - 4, F + 4, 0, 8, 4, H, F)[15] == 0
        assert orc.f32_rect_planes(5, 6, 0, 8, 4, H, F)[15] == 0


@pytest.mark.parametrize("F,tile", [(8, 8), (12, 8), (16, 16), (6, 4), (40, 8), (24, 4)])
def test_binning_is_conservative(orc, F, tile):
    sc = _scene_with_flat_and_tiny(14)
    o = np.float32([0.1, -0.1, 0.2])
    radii = scenes.radii_linear(0.1, 8, 8)
    with orc.atlas_map(1):
        keys, vals = orc.f32_bin(sc, o[None], 6 * F, F, radii, eps=1e-7, tile=tile)
        need = _brute_lists(orc, sc, o, 6 * F, F, tile, radii, 1e-7)
    got = set()
    for k, v in zip(keys.tolist(), vals.tolist()):
        for h in (0, 1):
            if (v >> (30 + h)) & 1:
                got.add((k, v & IDX, h))
    assert need <= got, sorted(need - got)[:5]
    if F % tile == 0:   # no tile across two faces (those take every Gaussian): the culling still culls
        assert len(got) < 3 * len(need) + 200
    order = np.lexsort((vals & IDX, keys))
    assert np.array_equal(order, np.arange(keys.size))


def test_roi_covers_the_box_receivers_and_marks_only_their_taps(orc):
    occ = scenes.cube_scene(400, seed=0)
    recv = scenes.cube_scene(3000, seed=1)
    lights = np.float32([[0, 0, 0], [0.8, 0.5, 1.2]])
    radii = scenes.radii_geometric(0.2, 9.0, 10)
    box = np.float32([0.3, -0.4, 1.1, 2.0, 4.2])
    F = 12
    H, K = 6 * F, radii.shape[0]
    p = recv.means
    inside = (np.abs(p[:, 0] - box[0]) <= box[2]) & (np.abs(p[:, 1] - box[1]) <= box[2]) & \
             (p[:, 2] >= box[3]) & (p[:, 2] <= box[4])
    with orc.atlas_map(1):
        dense = orc.build_atlas(occ, lights, H, F, radii)
        mask, kr = orc.f32_roi(p, box, lights, H, F, radii)
        roi = orc.roi_atlas(dense, mask, kr)
        _, T_d = orc.attenuate(dense, radii, lights, p[inside], recv.colors[inside], want_T=True)
        _, T_r = orc.attenuate(roi, radii, lights, p[inside], recv.colors[inside], want_T=True)
        assert np.array_equal(T_r, T_d) and dense.min() < 0.9
        for l in range(2):
            oi, of = orc.f32_sample_index(p[inside], lights[l], H, F, radii)
            oi = oi[of[:, 2] != 0]
            lo = (oi[:, 0] // F) * F
            ref = np.zeros((H, F), np.uint8)
            for di in (0, 1):
                for dj in (0, 1):
                    ref[np.clip(oi[:, 2] + di, lo, lo + F - 1), np.clip(oi[:, 3] + dj, 0, F - 1)] = 1
            assert np.array_equal(mask[l], ref)
    assert mask.mean() < 0.6
