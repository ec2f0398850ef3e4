"""Pins of the oracle's octahedral map (Eq. 6 and its inverse), its FP32 index
specification, the tile-binning specification (occluder culling, Sec. 3.2)
and the centre-sample lookup (Sec. 3.3)."""
import math

import numpy as np
import pytest

from paper_2601_01660_b300 import scenes


def test_encode_known_directions(orc):
    cases = {(0, 0, 1): (0, 0), (1, 0, 0): (1, 0), (0, 1, 0): (0, 1), (-1, 0, 0): (-1, 0),
             (0, -1, 0): (0, -1)}
    for d, uv in cases.items():
        assert orc.octa_encode(np.array(d, float)) == pytest.approx(uv, abs=1e-15)
    # -z folds onto the four corners; sgn(0) = +1 picks (+1,+1)
    assert orc.octa_encode(np.array([0, 0, -1.0])) == pytest.approx((1, 1))
    assert orc.octa_encode(np.array([1e-9, -1e-9, -1.0])) == pytest.approx((1, -1), abs=1e-8)


def test_encode_decode_inverse(orc):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        u, v = orc.octa_encode(d)
        assert -1 <= u <= 1 and -1 <= v <= 1
        np.testing.assert_allclose(orc.octa_decode(u, v), d, atol=1e-14)
        uv = rng.uniform(-1, 1, 2)
        dd = orc.octa_decode(*uv)
        assert np.linalg.norm(dd) == pytest.approx(1.0, abs=1e-15)
        np.testing.assert_allclose(orc.octa_encode(dd), uv, atol=1e-14)


@pytest.mark.parametrize("H,W", [(64, 64), (256, 256), (512, 512), (48, 80)])
def test_f32_round_trip_every_texel(orc, H, W):
    """encode(decode(texel centre)) lands in the same texel under the FP32 spec."""
    dirs = np.array([orc.texel_dir(i, j, H, W) for i in range(H) for j in range(W)])
    pts = (dirs * 3.0).astype(np.float32)
    ints, fl = orc.f32_sample_index(pts, np.zeros(3), H, W, scenes.radii_linear(0.1, 8, 4))
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    assert np.array_equal(ints[:, 0], ii.ravel())
    assert np.array_equal(ints[:, 1], jj.ravel())
    # the bilinear base sits on the texel itself (fraction ~0) or its lower
    # neighbour (fraction ~1) when rounding lands a hair below the centre
    fx = fl[:, 1]
    near0 = (ints[:, 3] == jj.ravel()) & (fx < 1e-3)
    near1 = (ints[:, 3] == jj.ravel() - 1) & (fx > 1 - 1e-3)
    assert np.all(near0 | near1)


def test_f32_index_agrees_with_fp64_encode(orc):
    rng = np.random.default_rng(1)
    H, W = 96, 128
    radii = scenes.radii_geometric(0.05, 12, 20)
    o = np.float32([0.3, -0.2, 1.0])
    pts = np.float32(rng.uniform(-6, 6, (3000, 3)))
    ints, fl = orc.f32_sample_index(pts, o, H, W, radii)
    for p, iv, fv in zip(pts, ints, fl):
        v = p.astype(np.float64) - o
        t = np.linalg.norm(v)
        u, vv = orc.octa_encode(v / t)
        gx = (u + 1) / 2 * W - 0.5
        gy = (vv + 1) / 2 * H - 0.5
        assert iv[3] + fv[1] == pytest.approx(gx, abs=2e-4)
        assert iv[2] + fv[0] == pytest.approx(gy, abs=2e-4)
        k = int(np.sum(radii.astype(np.float64) <= t)) - 1
        assert abs(iv[4] - k) <= 1 and fv[2] == pytest.approx(t, rel=1e-6)


@pytest.mark.parametrize("H,W,tile", [(64, 64, 8), (44, 60, 8), (128, 128, 16), (40, 40, 4)])
def test_tile_cones_contain_their_texels(orc, H, W, tile):
    for i0 in range(0, H, tile):
        for j0 in range(0, W, tile):
            i1, j1 = min(i0 + tile, H), min(j0 + tile, W)
            cone = orc.f32_rect_cone(i0, i1, j0, j1, H, W)
            if cone[5]:
                continue
            c = cone[:3].astype(np.float64)
            for i in range(i0, i1):
                for j in range(j0, j1):
                    d = orc.texel_dir(i, j, H, W)
                    assert d @ c >= cone[3] - 1e-6


def test_gauss_cone_bounds_the_culling_ellipsoid(orc):
    """Every point of the k-ellipsoid {(x-mu)^T A (x-mu) <= k^2} lies inside the
    cone (and the sphere) the binning spec gives the Gaussian."""
    sc = scenes.cube_scene(200, seed=12)
    o = np.float32([0.2, 0.1, 0.0])
    rng = np.random.default_rng(2)
    for i in range(sc.n):
        r, g = orc.f32_gauss_cone(sc.means[i], sc.scales[i], sc.opac[i], o, 1.0, 1e-7, 8.0)
        assert r in (0, 1)
        if r == 0 or g[5]:
            continue
        k = math.sqrt(g[6])
        R = orc.rotation(sc.quats[i])
        z = rng.normal(size=(64, 3))
        z /= np.linalg.norm(z, axis=1, keepdims=True)
        pts = sc.means[i] + (z * k * sc.scales[i]) @ R.T
        v = pts - o
        cosang = (v / np.linalg.norm(v, axis=1, keepdims=True)) @ g[:3].astype(np.float64)
        assert np.all(cosang >= g[3] - 1e-6)


def test_cull_radius_bounds_missed_optical_depth(orc):
    """A ray that misses the k-ellipsoid carries at most eps of optical depth
    from that Gaussian: beta I(inf) <= kappa odds (s_max/s_min) e^{-k^2/2} <= eps."""
    rng = np.random.default_rng(4)
    sc = scenes.cube_scene(60, seed=13)
    eps = 1e-7
    for i in range(sc.n):
        r, g = orc.f32_gauss_cone(sc.means[i], sc.scales[i], sc.opac[i], np.zeros(3), 1.0, eps, 1e9)
        k = math.sqrt(g[6])
        A = orc.precision(sc.scales[i], sc.quats[i])
        Rm = orc.rotation(sc.quats[i])
        one = scenes.subset(sc, [i])
        for _ in range(10):
            # aim at a point just outside the ellipsoid (Mahalanobis radius 1.02 k)
            z = rng.normal(size=3)
            z /= np.linalg.norm(z)
            p = sc.means[i] + Rm @ (z * 1.02 * k * sc.scales[i])
            d = p / np.linalg.norm(p)
            a, b, c = orc.ray_coeffs(A, d, -sc.means[i].astype(np.float64))
            m2 = c - b * b / a
            if m2 < k * k:   # this ray still cuts the ellipsoid elsewhere
                continue
            tau = orc.tau_rays(one, np.zeros((1, 3)), d[None], [1e4])[0]
            assert tau <= eps * 1.0001


IDX = 0x3FFFFFFF   # Gaussian index bits of a pair value; bits 30, 31: half-tile mask


def _brute_lists(orc, sc, o, H, W, tile, radii, eps):
    """Which (tile, Gaussian, half) triples must be binned: some texel ray of
    the tile's half (rows [0, tile/2) or [tile/2, tile)) cuts the Gaussian's
    k-ellipsoid at t > 0 within the shells (FP64)."""
    ty, tx = -(-H // tile), -(-W // tile)
    need = set()
    dirs = np.array([[orc.texel_dir(i, j, H, W) for j in range(W)] for i in range(H)])
    for g in range(sc.n):
        r, cone = orc.f32_gauss_cone(sc.means[g], sc.scales[g], sc.opac[g], o, 1.0, eps,
                                     float(radii[-1]))
        if r != 1:
            continue
        k2 = float(cone[6])
        A = orc.precision(sc.scales[g], sc.quats[g])
        om = o.astype(np.float64) - sc.means[g]
        Ad = dirs @ A            # (H,W,3)
        a = np.einsum("hwc,hwc->hw", Ad, dirs)
        b = Ad @ om
        c = om @ A @ om
        m2 = c - b * b / a
        hit = (m2 <= k2) & (-b / a > 0)
        for i, j in zip(*np.nonzero(hit)):
            need.add(((i // tile) * tx + (j // tile), g, int(i % tile >= tile // 2)))
    return need


def _scene_with_flat_and_tiny(seed):
    """Anisotropic cube Gaussians, flat surface Gaussians (2 mm thick) and
    tiny avatar Gaussians: the shapes the ellipsoid test must bound."""
    rng = np.random.default_rng(seed)
    a = scenes.cube_scene(90, seed=seed, log_s_mean=math.log(0.08))
    f = scenes.cube_scene(90, seed=seed + 1, log_s_mean=math.log(0.15))
    f.scales[:, rng.integers(0, 3, f.n)] = 0.002
    f.scales[np.arange(f.n), rng.integers(0, 3, f.n)] = 0.002
    t = scenes.avatar_body(rng, 60, base=(0.0, 0.5, 1.0))
    return scenes.concat(a, f, t)


@pytest.mark.parametrize("H,W,tile", [(32, 32, 8), (40, 56, 8), (44, 40, 8), (64, 64, 16), (36, 28, 4)])
def test_binning_is_conservative(orc, H, W, tile):
    sc = _scene_with_flat_and_tiny(14)
    o = np.float32([0.1, -0.1, 0.2])
    radii = scenes.radii_linear(0.1, 8, 8)
    keys, vals = orc.f32_bin(sc, o[None], H, W, radii, eps=1e-7, tile=tile)
    got = set()
    for k, v in zip(keys.tolist(), vals.tolist()):
        for h in (0, 1):
            if (v >> (30 + h)) & 1:
                got.add((k, v & IDX, h))
    need = _brute_lists(orc, sc, o, H, W, tile, radii, 1e-7)
    assert need <= got, sorted(need - got)[:5]
    # the lists come out ordered by (key, Gaussian index); every pair has a half
    order = np.lexsort((vals & IDX, keys))
    assert np.array_equal(order, np.arange(keys.size))
    assert np.all(vals >> 30 != 0)


def test_ellipsoid_test_trims_a_flat_gaussian(orc):
    """A 2 mm thick disc seen edge-on: its bounding sphere's cone covers a
    disc of tiles, its ellipsoid only a thin band of them."""
    H = W = 256
    tile = 8
    sc = scenes.Scene(np.float32([[0.0, 0.0, 3.0]]), np.float32([[0.3, 0.3, 0.002]]),
                      np.float32([[np.cos(np.pi / 4), np.sin(np.pi / 4), 0.0, 0.0]]), np.float32([0.9]),
                      np.float32([[1, 1, 1]]))
    o = np.float32([0, 0, 0])
    keys, vals = orc.f32_bin(sc, o[None], H, W, scenes.radii_linear(0.1, 8, 8), tile=tile)
    r, g = orc.f32_gauss_cone(sc.means[0], sc.scales[0], sc.opac[0], o, 1.0, 1e-7, 8.0)
    tx = W // tile
    sphere = 0
    for t in range(tx * tx):
        ti, tj = divmod(t, tx)
        c = orc.f32_rect_cone(ti * tile, ti * tile + tile, tj * tile, tj * tile + tile, H, W)
        sphere += float(g[:3] @ c[:3]) >= float(g[3] * c[3] - g[4] * c[4])
    assert sphere > 40 and len(keys) < 0.5 * sphere


def test_rect_planes_bound_their_texels(orc):
    """Every texel-centre direction of a valid rectangle is on the
    non-negative side of its four edge planes and on the correct side of the
    mid plane; a rectangle across the fold of the octahedral map (or one row
    high) has no planes."""
    H, W = 48, 64
    for (i0, i1, j0, j1) in [(0, 8, 0, 8), (16, 24, 40, 48), (40, 48, 56, 64), (8, 16, 24, 32), (3, 11, 5, 13)]:
        pl = orc.f32_rect_planes(i0, i1, j0, j1, 4, H, W)
        if pl[15] == 0:
            continue
        for i in range(i0, i1):
            for j in range(j0, j1):
                d = orc.texel_dir(i, j, H, W)
                for q in range(4):
                    assert pl[3 * q: 3 * q + 3] @ d >= -1e-6
                side = pl[12:15] @ d
                assert (side >= -1e-6) if i < i0 + 4 else (side <= 1e-6)
    # a tile that straddles |u| + |v| = 1 and a one-row tile
    assert orc.f32_rect_planes(20, 28, 52, 60, 4, H, W)[15] == 0
    assert orc.f32_rect_planes(5, 6, 0, 8, 4, H, W)[15] == 0


def test_gauss_axes_give_the_covariance(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        s = np.float32(np.exp(rng.normal(-3, 1, 3)))
        q = np.float32(rng.standard_normal(4))
        mu, o = np.float32(rng.normal(size=3)), np.float32(rng.normal(size=3))
        ax = orc.f32_gauss_axes(mu, s, q, o)
        C = ax[3:].reshape(3, 3).astype(np.float64)     # rows: s_k r_k
        A = orc.precision(s, q / np.linalg.norm(q))
        np.testing.assert_allclose(C.T @ C, np.linalg.inv(A), rtol=1e-4, atol=1e-6 * np.max(s) ** 2)
        np.testing.assert_allclose(ax[:3], mu.astype(np.float64) - o, rtol=1e-6, atol=1e-7)


def test_binned_sum_matches_full_sum(orc):
    """Summing Eq. 3 over the binned Gaussians only (per half tile) changes
    tau by at most (number of Gaussians) x eps per voxel."""
    sc = _scene_with_flat_and_tiny(15)
    o = np.float32([0, 0, 0])
    H = W = 16
    tile = 8
    radii = scenes.radii_linear(0.1, 8, 6)
    eps = 1e-7
    keys, vals = orc.f32_bin(sc, o[None], H, W, radii, eps=eps, tile=tile)
    full = orc.build_tau(sc, o[None], H, W, radii)[0]
    tx = W // tile
    for t in range((H // tile) * (W // tile)):
        ti, tj = divmod(int(t), tx)
        for h in (0, 1):
            sel = (keys == t) & (((vals >> (30 + h)) & 1) == 1)
            r0 = ti * tile + h * tile // 2
            blk = (slice(None), slice(r0, r0 + tile // 2), slice(tj * tile, tj * tile + tile))
            if sel.any():
                part = orc.build_tau(scenes.subset(sc, vals[sel] & IDX), o[None], H, W, radii)[0]
                assert np.max(np.abs(part[blk] - full[blk])) <= sc.n * eps
            else:
                assert np.max(full[blk]) <= sc.n * eps


def test_sample_at_voxel_centre_returns_voxel(orc):
    rng = np.random.default_rng(7)
    K, H, W = 5, 12, 20
    radii = scenes.radii_geometric(0.2, 9.0, K)
    atlas = rng.random((K, H, W))
    o = np.array([0.5, -0.25, 1.0])
    for _ in range(50):
        k, i, j = rng.integers(K), rng.integers(H), rng.integers(W)
        x = o + orc.texel_dir(i, j, H, W) * float(radii[k])
        assert orc.sample_T(atlas, radii, o, x) == pytest.approx(atlas[k, i, j], abs=1e-9)


def test_sample_is_trilinear(orc):
    """An atlas linear in (j, i, r) is reproduced exactly between texel centres
    and bracketing shells (away from the clamped borders and the fold)."""
    K, H, W = 6, 32, 32
    radii = scenes.radii_linear(0.5, 5.5, K)
    kk, ii, jj = np.meshgrid(np.arange(K), np.arange(H), np.arange(W), indexing="ij")
    atlas = 0.01 * jj + 0.02 * ii + 0.1 * radii.astype(np.float64)[kk]
    rng = np.random.default_rng(8)
    o = np.zeros(3)
    for _ in range(300):
        u, v = rng.uniform(-0.45, 0.45, 2)      # inside the upper diamond
        d = orc.octa_decode(u, v)
        t = rng.uniform(0.6, 5.4)
        gx = (u + 1) / 2 * W - 0.5
        gy = (v + 1) / 2 * H - 0.5
        ref = 0.01 * gx + 0.02 * gy + 0.1 * t
        assert orc.sample_T(atlas, radii, o, d * t) == pytest.approx(ref, abs=1e-9)


def test_attenuate_weights_and_direct_fraction(orc):
    rng = np.random.default_rng(9)
    L, K, H, W = 3, 4, 8, 8
    radii = scenes.radii_linear(0.1, 8, K)
    atlas = np.empty((L, K, H, W))
    for l, val in enumerate([0.2, 0.5, 0.9]):
        atlas[l] = val
    lights = np.float32([[0, 0, 0], [1, 0, 0], [0, 1, 0]])
    qm = np.float32(rng.uniform(-3, 3, (10, 3)))
    col = np.float32(rng.random((10, 3)))
    c64 = col.astype(np.float64)
    out = orc.attenuate(atlas, radii, lights, qm, col)
    np.testing.assert_allclose(out, c64 * (0.2 + 0.5 + 0.9) / 3, rtol=1e-12)
    out = orc.attenuate(atlas, radii, lights, qm, col, light_w=np.float32([1, 0, 0]),
                        direct_frac=0.5)
    np.testing.assert_allclose(out, c64 * (0.5 + 0.5 * 0.2), rtol=1e-7)
    out, T = orc.attenuate(atlas, radii, lights, qm, col, atlas_dyn=atlas, want_T=True)
    np.testing.assert_allclose(T, np.tile([0.04, 0.25, 0.81], (10, 1)), rtol=1e-12)


def _room_like_scene(seed):
    """The room's shapes at a size the brute force covers: 2 mm floor discs
    3-5 m from a light 2.8 m above the floor, wall discs up to the height of
    the light (their rays cross the fold |u| + |v| = 1 of the octahedral map)
    and small avatar Gaussians."""
    rng = np.random.default_rng(seed)
    n_f, n_w = 120, 90
    r = rng.uniform(1.8, 4.0, n_f)
    phi = rng.uniform(0, 2 * np.pi, n_f)
    floor_m = np.stack([r * np.cos(phi), r * np.sin(phi), np.zeros(n_f)], 1)
    floor_s = np.stack([np.exp(rng.normal(math.log(0.05), 0.5, n_f)),
                        np.exp(rng.normal(math.log(0.05), 0.5, n_f)), np.full(n_f, 0.002)], 1)
    yaw = rng.uniform(0, np.pi, n_f)
    floor_q = np.stack([np.cos(yaw / 2), np.zeros(n_f), np.zeros(n_f), np.sin(yaw / 2)], 1)
    wall_m = np.stack([np.full(n_w, 4.0), rng.uniform(-3, 3, n_w), rng.uniform(2.0, 3.0, n_w)], 1)
    wall_s = np.stack([np.full(n_w, 0.002), np.exp(rng.normal(math.log(0.05), 0.5, n_w)),
                       np.exp(rng.normal(math.log(0.05), 0.5, n_w))], 1)
    wall_q = np.tile([1.0, 0.0, 0.0, 0.0], (n_w, 1))
    n = n_f + n_w
    room = scenes.Scene(np.float32(np.concatenate([floor_m, wall_m])), np.float32(np.concatenate([floor_s, wall_s])),
                        np.float32(np.concatenate([floor_q, wall_q])), np.float32(rng.uniform(0.05, 0.95, n)),
                        np.float32(rng.random((n, 3))))
    return scenes.concat(room, scenes.avatar_body(rng, 60, base=(1.5, 0.0, 0.0)))


def test_binning_is_conservative_room_shapes(orc):
    sc = _room_like_scene(21)
    o = np.float32([0.0, 0.0, 2.8])
    radii = scenes.radii_geometric(0.05, 12, 16)
    H = W = 96
    tile = 8
    keys, vals = orc.f32_bin(sc, o[None], H, W, radii, eps=1e-7, tile=tile)
    got = set()
    for k, v in zip(keys.tolist(), vals.tolist()):
        for h in (0, 1):
            if (v >> (30 + h)) & 1:
                got.add((k, v & IDX, h))
    need = _brute_lists(orc, sc, o, H, W, tile, radii, 1e-7)
    assert len(need) > 300
    assert need <= got, sorted(need - got)[:5]
    # some of the needed pairs lie on tiles across the octahedral fold
    tx = W // tile
    fold = 0
    for (t, g, h) in need:
        ti, tj = divmod(t, tx)
        u = [(2 * (tj * tile + d) + 1) / W - 1 for d in (0, tile - 1)]
        v = [(2 * (ti * tile + d) + 1) / H - 1 for d in (0, tile - 1)]
        s = [abs(a) + abs(b) for a in u for b in v]
        fold += min(s) < 1 < max(s)
    assert fold > 0


def test_binned_sum_matches_full_sum_room_shapes(orc):
    sc = _room_like_scene(22)
    o = np.float32([0.0, 0.0, 2.8])
    H = W = 48
    tile = 8
    radii = scenes.radii_geometric(0.05, 12, 12)
    eps = 1e-7
    keys, vals = orc.f32_bin(sc, o[None], H, W, radii, eps=eps, tile=tile)
    full = orc.build_tau(sc, o[None], H, W, radii)[0]
    tx = W // tile
    worst = 0.0
    for t in range((H // tile) * (W // tile)):
        ti, tj = divmod(int(t), tx)
        for h in (0, 1):
            sel = (keys == t) & (((vals >> (30 + h)) & 1) == 1)
            r0 = ti * tile + h * tile // 2
            blk = (slice(None), slice(r0, r0 + tile // 2), slice(tj * tile, tj * tile + tile))
            part = (orc.build_tau(scenes.subset(sc, vals[sel] & IDX), o[None], H, W, radii)[0][blk]
                    if sel.any() else 0.0)
            worst = max(worst, float(np.max(np.abs(part - full[blk]))))
    assert worst <= sc.n * eps
    assert full.max() > 0.5   # the sample holds real shadow


def test_bin_keys_is_the_specification_on_its_tiles(orc):
    """The tile-filtered binning (used at full size) returns exactly the full
    specification's pairs of the requested tiles."""
    rng = np.random.default_rng(23)
    sc = _room_like_scene(23)
    lights = np.float32([[0.0, 0.0, 2.8], [1.0, 1.0, 2.5]])
    radii = scenes.radii_geometric(0.05, 12, 16)
    for H, W, tile in [(64, 64, 8), (40, 56, 8), (64, 48, 16), (36, 28, 4)]:
        ko, vo = orc.f32_bin(sc, lights, H, W, radii, tile=tile)
        nt = -(-H // tile) * -(-W // tile)
        want = rng.choice(2 * nt, min(60, 2 * nt), replace=False)
        ks, vs = orc.f32_bin_keys(sc, lights, H, W, radii, want, tile=tile)
        m = np.isin(ko, want)
        assert ks.size > 0
        assert np.array_equal(ks, ko[m]) and np.array_equal(vs, vo[m])
