"""GPU parity of the per-frame mechanics for moving avatars: the capacity
(non-blocking) build, rigid motion, per-object centroids and relight,
attenuation by a static times a dynamic atlas of its own shape, graph
capture and replay of a whole frame, and the build autotuner."""
import numpy as np
import pytest
import torch

from oracle import motion
from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev, texel_sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _small_build_inputs(n=3000, seed=4):
    sc = scenes.cube_scene(n, seed=seed)
    lights = np.float32([[0, 0, 0], [0.5, -0.4, 0.8]])
    radii = scenes.radii_geometric(0.05, 9, 12)
    return sc, lights, radii


def test_capacity_build_equals_exact_build(nat):
    sc, lights, radii = _small_build_inputs()
    d = scene_to_dev(sc)
    args = (d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 48, 64, dev(radii))
    exact = nat.dgsm_build(*args)
    P = nat.dgsm_get_build_stats()["n_pairs"]
    assert P > 1000
    for cap in (P, 2 * P + 17):
        a = nat.dgsm_build(*args, params=dict(max_pairs=cap))
        assert nat.dgsm_sync_status() == 0
        assert nat.dgsm_get_build_stats()["n_pairs"] == P
        assert torch.allclose(a, exact, atol=1e-6, rtol=0)


def test_capacity_overflow_is_reported_and_safe(nat):
    sc, lights, radii = _small_build_inputs()
    d = scene_to_dev(sc)
    args = (d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 48, 64, dev(radii))
    nat.dgsm_build(*args)
    P = nat.dgsm_get_build_stats()["n_pairs"]
    a = nat.dgsm_build(*args, params=dict(max_pairs=P // 3))
    assert nat.dgsm_sync_status() == 3          # DGSM_ERR_WORKSPACE
    assert bool((a == 1.0).all())              # no pairs kept: unshadowed
    assert nat.dgsm_sync_status() == 0
    b = nat.dgsm_build(*args, params=dict(max_pairs=P))
    assert nat.dgsm_sync_status() == 0 and float(b.min()) < 0.5


def test_rigid_transform_matches_oracle(nat):
    rng = np.random.default_rng(1)
    rest, seg, _ = scenes.avatar_crowd(seed=3, n_avatars=5, n_each=2001)
    seg = [0, 2001, 2001 * 2, 2001 * 2 + 7, 2001 * 4, 2001 * 5]  # uneven objects
    poses = np.float32(np.concatenate([rng.standard_normal((5, 4)), rng.uniform(-3, 3, (5, 3)),
                                       np.zeros((5, 1))], 1))
    m, q = nat.dgsm_rigid_transform(dev(rest.means), dev(rest.quats), seg, dev(poses))
    mr, qr = motion.rigid_transform(rest.means, rest.quats, seg, poses)
    np.testing.assert_allclose(m.cpu().numpy(), mr, atol=2e-6, rtol=0)
    np.testing.assert_allclose(q.cpu().numpy(), qr, atol=2e-6, rtol=0)
    # poses from pinned host memory, in place
    mm, qq = dev(rest.means), dev(rest.quats)
    nat.dgsm_rigid_transform(mm, qq, seg, torch.as_tensor(poses).pin_memory(), means_out=mm, quats_out=qq)
    assert torch.equal(mm, m) and torch.equal(qq, q)


def test_segment_centroids_match_oracle(nat):
    sc = scenes.cube_scene(50_000, seed=2)
    seg = [0, 1, 20_000, 20_000, 50_000]
    c = nat.dgsm_segment_centroids(dev(sc.means), dev(sc.opac), seg)
    ref = motion.segment_centroids(sc.means, sc.opac, seg)
    np.testing.assert_allclose(c.cpu().numpy(), ref, atol=1e-6)
    c1 = nat.dgsm_segment_centroids(dev(sc.means), None, [0, sc.n])
    np.testing.assert_allclose(c1.cpu().numpy()[0], sc.means.astype(np.float64).mean(0), atol=1e-6)


def test_relight_objects_equals_per_object_relight(nat, orc):
    rest, seg, mo = scenes.avatar_crowd(seed=5, n_avatars=3, n_each=4000)
    poses = scenes.avatar_poses(mo, 17)
    d = scene_to_dev(rest)
    m, q = nat.dgsm_rigid_transform(d["means"], d["quats"], seg, dev(poses))
    cen = nat.dgsm_segment_centroids(m, d["opac"], seg)
    D, Y, w = scenes.cubemap_samples(16, seed=5)
    sh = nat.sh_fit(dev(D), dev(Y), dev(w))
    out = nat.sh_relight_objects(sh, m, q, d["scales"], d["colors"], cen, seg)
    shd = sh.double().cpu().numpy()
    for o in range(3):
        a, b = seg[o], seg[o + 1]
        one = nat.sh_relight(sh, m[a:b], q[a:b], d["scales"][a:b], d["colors"][a:b], cen[o])
        assert torch.equal(out[a:b], one)
        moved = scenes.Scene(m[a:b].cpu().numpy(), rest.scales[a:b], q[a:b].cpu().numpy(),
                             rest.opac[a:b], rest.colors[a:b])
        ref = orc.relight(shd, moved, cen[o].cpu().numpy())
        err = np.abs(one.double().cpu().numpy() - ref) / np.maximum(np.abs(ref), 1e-6)
        assert np.quantile(err, 0.999) <= 1e-3


def test_attenuate_dyn_matches_oracle(nat, orc):
    rng = np.random.default_rng(7)
    L = 3
    radii, radii_d = scenes.radii_geometric(0.1, 9, 10), scenes.radii_linear(0.2, 7, 5)
    atlas = np.sort(rng.random((L, 10, 40, 36)), axis=1)[:, ::-1].copy()
    dyn = np.sort(rng.random((L, 5, 17, 23)), axis=1)[:, ::-1].copy()
    lights = np.float32([[0, 0, 0], [1, -0.5, 0.5], [-2, 1, 3]])
    qm = np.float32(rng.uniform(-9, 9, (40_000, 3)))
    qm[:10] = lights[1]
    col = np.float32(rng.random((40_000, 3)))
    lw = np.float32([0.5, 0.2, 0.3])
    out, T = nat.dgsm_attenuate_dyn(dev(atlas), dev(radii), dev(dyn), dev(radii_d), dev(lights), dev(qm),
                                    dev(col), light_w=dev(lw), direct_frac=0.8, want_T=True)
    ref, Tref = motion.attenuate_two(np.float32(atlas), radii, np.float32(dyn), radii_d, lights, qm, col,
                                     light_w=lw, direct_frac=0.8)
    assert np.abs(T.double().cpu().numpy() - Tref).max() <= 1e-5
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 1e-5


@pytest.fixture(scope="module")
def crowd(nat):
    from paper_2601_01660_b300.frame import CrowdFrame
    wl = scenes.workload("crowd8s")
    D, Y, w = wl["cubemap"]
    sh = nat.sh_fit(dev(D), dev(Y), dev(w))
    cf = CrowdFrame(wl["static"], wl["avatars"], wl["seg"], wl["lights"], wl["H"], wl["W"], wl["radii"],
                    wl["H_dyn"], wl["W_dyn"], wl["radii_dyn"], sh)
    cf.size_pairs([scenes.avatar_poses(wl["motion"], f) for f in range(0, 120, 20)])
    yield wl, cf
    cf.close()


def test_dynamic_atlas_matches_oracle(nat, orc, crowd):
    wl, cf = crowd
    poses = scenes.avatar_poses(wl["motion"], 33)
    cf.step_eager(poses, max_pairs=cf.max_pairs)
    cf.stream.synchronize()
    assert nat.dgsm_sync_status(cf.ctx) == 0
    av = wl["avatars"]
    mr, qr = motion.rigid_transform(av.means, av.quats, wl["seg"], poses)
    moved = scenes.Scene(np.float32(mr), av.scales, np.float32(qr), av.opac, av.colors)
    lij = texel_sample(np.random.default_rng(3), 4, cf.H_dyn, cf.W_dyn, 24)
    tau = orc.build_tau_texels(moved, wl["lights"], cf.H_dyn, cf.W_dyn, wl["radii_dyn"], lij)
    got = cf.dyn_atlas.double().cpu().numpy()[lij[:, 0], :, lij[:, 1], lij[:, 2]]
    assert np.abs(got - np.exp(-tau)).max() <= 1e-4


def test_graph_replay_equals_eager_frames(nat, crowd):
    wl, cf = crowd
    n_nodes = cf.capture()
    assert n_nodes > 10
    for f in (5, 6, 7, 90):
        poses = scenes.avatar_poses(wl["motion"], f)
        cf.step_graph(poses)
        cf.stream.synchronize()
        assert nat.dgsm_sync_status(cf.ctx) == 0
        g_out, g_atl = cf.colors_out.clone(), cf.dyn_atlas.clone()
        torch.cuda.synchronize()
        cf.step_eager(poses)
        cf.stream.synchronize()
        assert torch.allclose(cf.dyn_atlas, g_atl, atol=1e-6, rtol=0)
        assert torch.allclose(cf.colors_out, g_out, atol=1e-5, rtol=1e-5)
    # the avatars moved between frames
    a0 = scenes.avatar_poses(wl["motion"], 5)[:, 4:7]
    a1 = scenes.avatar_poses(wl["motion"], 90)[:, 4:7]
    assert np.abs(a0 - a1).max() > 0.5


def test_workspace_is_frozen_while_a_graph_lives(nat, crowd):
    wl, cf = crowd
    if cf.graphs is None:
        cf.capture()
    big = scenes.cube_scene(4 * cf.n_dyn, seed=9)
    d = scene_to_dev(big)
    # a build needing more workspace than the graphs were captured with fails
    # cleanly, before it launches anything
    with pytest.raises(nat.DGSMError):
        nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], cf.lights, cf.H_dyn, cf.W_dyn,
                       cf.radii_dyn, ctx=cf.ctx, stream=cf.stream)
    cf.step_graph(scenes.avatar_poses(wl["motion"], 3))
    cf.stream.synchronize()
    assert nat.dgsm_sync_status(cf.ctx) == 0


def test_autotune_picks_a_measured_candidate(nat):
    sc, lights, radii = _small_build_inputs(n=4000)
    d = scene_to_dev(sc)
    best, table = nat.dgsm_autotune_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 64,
                                          64, dev(radii), tiles=(8, 16), chunks=(32, 128), reps=2)
    assert set(table) == {(8, 32), (8, 128), (16, 32), (16, 128)}
    ran = {k: v for k, v in table.items() if v >= 0}
    assert ran and (best.tile, best.chunk) == min(ran, key=ran.get)
