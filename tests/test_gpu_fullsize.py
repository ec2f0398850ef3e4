"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on outputs the FP64 oracle computes one by one (sampled texels,
queries and Gaussians), plus the largest sizes the API accepts and degenerate
Gaussians.  Collected after the per-feature GPU tests."""
import math

import numpy as np
import pytest
import torch

from oracle import motion
from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev, texel_sample

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-4


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


@pytest.fixture(scope="module")
def room(nat):
    """The room workload built and attenuated exactly as one bench step does."""
    wl = scenes.workload("room1p6m")
    sc = wl["occluders"]
    d = scene_to_dev(sc)
    lights, radii = dev(wl["lights"]), dev(wl["radii"])
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, wl["H"], wl["W"], radii)
    out, T = nat.dgsm_attenuate(atlas, radii, lights, d["means"], d["colors"], want_T=True)
    return wl, d, atlas, out, T


def test_room_build_sampled_texels(nat, orc, room):
    wl, d, atlas, _, _ = room
    lij = texel_sample(np.random.default_rng(11), 1, wl["H"], wl["W"], 16)
    lij[0] = (0, 255, 255)       # next to the direction straight down
    lij[1] = (0, 0, 0)           # a corner of the fold
    tau = orc.build_tau_texels(wl["occluders"], wl["lights"], wl["H"], wl["W"], wl["radii"], lij)
    got = atlas.double().cpu().numpy()[lij[:, 0], :, lij[:, 1], lij[:, 2]]
    err = np.abs(got - np.exp(-tau))
    assert err.max() <= TOL_F32, err.max()
    assert np.exp(-tau).min() < 0.5  # the sample sees real shadow


def _texel_of(orc, direction, H, W):
    """(row, column) of the texel holding a direction (row i <-> v, column j <-> u)."""
    u, v = orc.octa_encode(np.asarray(direction, dtype=np.float64))
    return min(max(int((v + 1) * 0.5 * H), 0), H - 1), min(max(int((u + 1) * 0.5 * W), 0), W - 1)


def test_room_build_shadow_texels(nat, orc, room):
    """256 texels of the room atlas against the FP64 brute force: the deepest
    shadows and the sharpest shadow edges the build found, the avatar's
    shadow, texels along the octahedral fold and at the map's corners (the
    direction straight down), and random ones."""
    wl, d, atlas, _, _ = room
    H, W = wl["H"], wl["W"]
    A = atlas[0].double().cpu().numpy()          # [K][H][W]
    rng = np.random.default_rng(14)
    last = A[-1]
    deep = np.argsort(last, axis=None)[:4000]
    edge = np.abs(np.diff(A[-1], axis=1))
    edges = np.argsort(edge, axis=None)[::-1][:4000]
    pick = list(rng.choice(deep, 64, replace=False))
    pick += [int(i * W + j) for i, j in zip(*np.unravel_index(rng.choice(edges, 64, replace=False), edge.shape))]
    o = wl["lights"][0].astype(np.float64)
    sl = wl["occluders"].meta["avatar"]
    av = wl["occluders"].means[sl].astype(np.float64)
    for p in av[rng.choice(len(av), 32, replace=False)]:
        i, j = _texel_of(orc, p - o, H, W)
        pick.append(i * W + j)
    fold = [(i, j) for i in range(H) for j in range(W)
            if abs(abs((2 * j + 1) / W - 1) + abs((2 * i + 1) / H - 1) - 1) < 2.0 / W]
    pick += [i * W + j for i, j in (fold[k] for k in rng.choice(len(fold), 32, replace=False))]
    pick += [0, W - 1, (H - 1) * W, H * W - 1]
    rest = 256 - len(set(pick))
    pick += list(rng.choice(H * W, rest + 16, replace=False))
    flat = np.array(sorted(set(int(x) for x in pick)))[:256]
    lij = np.stack([np.zeros_like(flat), flat // W, flat % W], 1).astype(np.int32)
    tau = orc.build_tau_texels(wl["occluders"], wl["lights"], H, W, wl["radii"], lij)
    got = A[:, lij[:, 1], lij[:, 2]].T
    err = np.abs(got - np.exp(-tau))
    assert lij.shape[0] == 256
    assert err.max() <= TOL_F32, err.max()
    assert np.exp(-tau).min() < 1e-3 and (np.exp(-tau)[:, -1] < 0.5).sum() >= 64


def test_room_binning_bit_exact_sampled_tiles(nat, orc, room):
    """The 512 x 512 room's tile lists equal the binning specification bit
    for bit on about 300 tiles: the longest lists, tiles across the fold,
    tiles toward the avatar, the corners, and random ones."""
    wl, d, _, _, _ = room
    H, W, tile = wl["H"], wl["W"], 8
    tx = W // tile
    kg, vg = nat.dgsm_bin(d["means"], d["scales"], d["quats"], d["opac"], dev(wl["lights"]), H, W,
                          dev(wl["radii"]))
    kg = kg.cpu().numpy().astype(np.uint32)
    vg = vg.cpu().numpy().astype(np.uint32)
    counts = np.bincount(kg, minlength=(H // tile) * tx)
    rng = np.random.default_rng(15)
    want = set(np.argsort(counts)[::-1][:60].tolist())
    for t in range(counts.size):
        ti, tj = divmod(t, tx)
        u = [(2 * (tj * tile + q) + 1) / W - 1 for q in (0, tile - 1)]
        v = [(2 * (ti * tile + q) + 1) / H - 1 for q in (0, tile - 1)]
        sums = [abs(a) + abs(b) for a in u for b in v]
        if min(sums) < 1 < max(sums) and rng.random() < 0.25:
            want.add(t)
    o = wl["lights"][0].astype(np.float64)
    sl = wl["occluders"].meta["avatar"]
    av = wl["occluders"].means[sl].astype(np.float64)
    for p in av[rng.choice(len(av), 40, replace=False)]:
        i, j = _texel_of(orc, p - o, H, W)
        want.add((i // tile) * tx + j // tile)
    want |= {0, tx - 1, counts.size - tx, counts.size - 1}
    for t in rng.permutation(counts.size).tolist():   # random tiles up to 300 in all
        if len(want) >= 300:
            break
        want.add(t)
    want = np.array(sorted(want), dtype=np.uint32)
    assert want.size == 300
    ko, vo = orc.f32_bin_keys(wl["occluders"], wl["lights"], H, W, wl["radii"], want)
    m = np.isin(kg, want)
    assert ko.size > 10 ** 6
    assert np.array_equal(kg[m], ko) and np.array_equal(vg[m], vo)


def test_room_attenuate_sampled_queries(nat, orc, room):
    wl, d, atlas, out, T = room
    sc = wl["occluders"]
    idx = np.random.default_rng(12).choice(sc.n, 3000, replace=False)
    ref, Tref = orc.attenuate(atlas.double().cpu().numpy(), wl["radii"], wl["lights"], sc.means[idx],
                              sc.colors[idx], want_T=True)
    # the FP32 texel coordinate carries ~3e-5 texel of rounding at 512 wide;
    # self-shadowed receivers sit where T changes by ~0.5 per texel and shell
    err_T = np.abs(T.double().cpu().numpy()[idx] - Tref)
    assert err_T.max() <= TOL_F32 and np.median(err_T) <= 1e-6
    assert np.abs(out.double().cpu().numpy()[idx] - ref).max() <= TOL_F32


def test_room_relight_sampled_gaussians(nat, orc, room):
    wl, d, atlas, out, _ = room
    sc = wl["occluders"]
    sl = sc.meta["avatar"]
    D, Y, w = wl["cubemap"]
    sh = nat.sh_fit(dev(D), dev(Y), dev(w))
    cen = nat.dgsm_weighted_centroid(d["means"][sl], d["opac"][sl])
    relit = nat.sh_relight(sh, d["means"][sl], d["quats"][sl], d["scales"][sl], out[sl], cen)
    av = scenes.subset(sc, np.arange(sl.start, sl.stop))
    pick = np.random.default_rng(13).choice(av.n, 1500, replace=False)
    sub = scenes.subset(av, pick)
    sub.colors = np.float32(out.cpu().numpy()[sl][pick])
    ref = orc.relight(sh.double().cpu().numpy(), sub, cen.cpu().numpy())
    got = relit.double().cpu().numpy()[pick]
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6)
    assert np.quantile(rel.max(1), 0.998) <= 1e-3   # a normal turned within rounding may differ


@pytest.mark.parametrize("persistent", [False, True])
def test_crowd_frame_full_size(nat, orc, persistent):
    """The 8-avatar frame at full size under graph replay, as separate calls
    and as the persistent frame kernel: the dynamic atlas on sampled texels
    and the final colours on sampled Gaussians."""
    from paper_2601_01660_b300.frame import CrowdFrame
    wl = scenes.workload("crowd8")
    D, Y, w = wl["cubemap"]
    sh = nat.sh_fit(dev(D), dev(Y), dev(w))
    cf = CrowdFrame(wl["static"], wl["avatars"], wl["seg"], wl["lights"], wl["H"], wl["W"], wl["radii"],
                    wl["H_dyn"], wl["W_dyn"], wl["radii_dyn"], sh, persistent=persistent)
    try:
        cf.size_pairs([scenes.avatar_poses(wl["motion"], f) for f in range(0, 120, 30)])
        cf.capture()
        poses = scenes.avatar_poses(wl["motion"], 47)
        cf.step_graph(poses)
        cf.stream.synchronize()
        assert nat.dgsm_sync_status(cf.ctx) == 0
        av, seg = wl["avatars"], wl["seg"]
        mr, qr = motion.rigid_transform(av.means, av.quats, seg, poses)
        moved = scenes.Scene(np.float32(mr), av.scales, np.float32(qr), av.opac, av.colors)
        lij = texel_sample(np.random.default_rng(14), 4, cf.H_dyn, cf.W_dyn, 12)
        tau = orc.build_tau_texels(moved, wl["lights"], cf.H_dyn, cf.W_dyn, wl["radii_dyn"], lij)
        got = cf.dyn_atlas.double().cpu().numpy()[lij[:, 0], :, lij[:, 1], lij[:, 2]]
        assert np.abs(got - np.exp(-tau)).max() <= TOL_F32
        # static receivers: colour = attenuation by static x dynamic atlases
        st = wl["static"]
        idx = np.random.default_rng(15).choice(st.n, 2000, replace=False)
        ref, _ = motion.attenuate_two(cf.static_atlas.double().cpu().numpy(), wl["radii"],
                                      cf.dyn_atlas.double().cpu().numpy(), wl["radii_dyn"], wl["lights"],
                                      st.means[idx], st.colors[idx])
        out = cf.colors_out.double().cpu().numpy()
        assert np.abs(out[idx] - ref).max() <= TOL_F32
        # avatars: attenuated, then relit around their own centroids
        ai = np.random.default_rng(16).choice(av.n, 800, replace=False)
        means_w = cf.av_means.cpu().numpy()
        att, _ = motion.attenuate_two(cf.static_atlas.double().cpu().numpy(), wl["radii"],
                                      cf.dyn_atlas.double().cpu().numpy(), wl["radii_dyn"], wl["lights"],
                                      means_w[ai], av.colors[ai])
        cen = motion.segment_centroids(means_w, av.opac, seg)
        obj = motion.object_of(seg, av.n)[ai]
        shd = sh.double().cpu().numpy()
        for o in np.unique(obj):
            sel = ai[obj == o]
            sub = scenes.Scene(means_w[sel], av.scales[sel], cf.av_quats.cpu().numpy()[sel], av.opac[sel],
                               np.float32(att[obj == o]))
            ref_o = orc.relight(shd, sub, cen[o])
            got_o = out[st.n + sel]
            rel = np.abs(got_o - ref_o) / np.maximum(np.abs(ref_o), 1e-6)
            assert np.quantile(rel.max(1), 0.99) <= 1e-3, (o, rel.max())
    finally:
        cf.close()


def test_largest_sizes(nat, orc):
    """K = 256 shells (every voxel) and a 4096 x 4096 atlas (sampled texels
    including the fold corners)."""
    sc = scenes.cube_scene(300, seed=21, log_s_mean=math.log(0.1))
    lights = np.float32([[0.1, 0.0, 0.2]])
    radii = scenes.radii_geometric(0.05, 9, 256)
    d = scene_to_dev(sc)
    T = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 12, 12, dev(radii),
                       params=dict(chunk=32)).double().cpu().numpy()
    assert np.abs(T - orc.build_atlas(sc, lights, 12, 12, radii)).max() <= TOL_F32
    radii = scenes.radii_linear(0.5, 8, 2)
    T = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 4096, 4096, dev(radii))
    lij = texel_sample(np.random.default_rng(22), 1, 4096, 4096, 60)
    corners = np.int32([[0, 0, 0], [0, 0, 4095], [0, 4095, 0], [0, 4095, 4095], [0, 2047, 2048], [0, 2048, 2047]])
    lij = np.concatenate([lij, corners])
    tau = orc.build_tau_texels(sc, lights, 4096, 4096, radii, lij)
    got = T.double().cpu().numpy()[lij[:, 0], :, lij[:, 1], lij[:, 2]]
    assert np.abs(got - np.exp(-tau)).max() <= TOL_F32


def test_degenerate_gaussians(nat, orc):
    """Needle- and sheet-like Gaussians (axis ratio 1e4), tiny and room-sized
    scales, near-opaque ones, one centred on the light and one the light sits
    inside: every voxel against the oracle."""
    rng = np.random.default_rng(23)
    n = 400
    sc = scenes.cube_scene(n, seed=24)
    sc.scales[:50] = np.float32([3e-4, 3.0, 0.3])          # sheets
    sc.scales[50:100] = np.float32([2.0, 2e-4, 2e-4])       # needles
    sc.scales[100:130] = 1e-4                               # tiny
    sc.scales[130:140] = 4.0                                # larger than the scene
    sc.opac[140:200] = 0.9999999                            # clamped to 1 - 1e-6
    sc.means[200] = 0.0                                     # at the light
    sc.means[201] = np.float32([0.1, 0.0, 0.0])
    sc.scales[201] = 0.5                                    # the light is inside it
    sc.quats[:] = np.float32(rng.standard_normal((n, 4)))   # un-normalised quaternions
    lights = np.float32([[0, 0, 0]])
    radii = scenes.radii_geometric(0.05, 10, 11)
    d = scene_to_dev(sc)
    for H, W in ((24, 24), (33, 47)):
        T = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W,
                           dev(radii)).double().cpu().numpy()
        err = np.abs(T - orc.build_atlas(sc, lights, H, W, radii))
        assert err.max() <= TOL_F32, err.max()
