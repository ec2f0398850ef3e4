"""GPU parity of the persistent frame kernel (dgsm_crowd_frame): one
cooperative launch per frame gives the frame of the separate calls (the
same motion, binned pairs and centroids exactly; the atlas and colours up
to the order of floating-point atomic sums), the dynamic atlas agrees with
the FP64 oracle, every grid barrier's bounded wait can be made to run out
and the context then builds again, an over-capacity frame is reported and
unshadowed, and the launch replays inside a CUDA graph."""
import numpy as np
import pytest
import torch

from oracle import motion
from paper_2601_01660_b300 import scenes

from gpu_util import dev, texel_sample

pytestmark = pytest.mark.gpu

DGSM_ERR_WORKSPACE, DGSM_ERR_TIMEOUT = 3, 4


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


@pytest.fixture(scope="module")
def pair(nat):
    """The small crowd twice, each on its own context: direct calls, and the
    persistent kernel with the same pair capacity."""
    from paper_2601_01660_b300.frame import CrowdFrame
    wl = scenes.workload("crowd8s")
    D, Y, w = wl["cubemap"]
    sh = nat.sh_fit(dev(D), dev(Y), dev(w))
    args = (wl["static"], wl["avatars"], wl["seg"], wl["lights"], wl["H"], wl["W"], wl["radii"], wl["H_dyn"],
            wl["W_dyn"], wl["radii_dyn"], sh)
    direct = CrowdFrame(*args, build_params=dict(tile=8))
    pers = CrowdFrame(*args, build_params=dict(tile=8), persistent=True)
    direct.size_pairs([scenes.avatar_poses(wl["motion"], f) for f in range(0, 120, 20)])
    pers.max_pairs = direct.max_pairs
    yield wl, direct, pers
    direct.close()
    pers.close()


def _run(nat, cf, poses, max_pairs=None):
    cf.step_eager(poses, max_pairs=cf.max_pairs if max_pairs is None else max_pairs)
    cf.stream.synchronize()
    return nat.dgsm_sync_status(cf.ctx)


def test_persistent_frame_equals_direct_calls(nat, pair):
    wl, direct, pers = pair
    for f in (3, 33, 77):
        poses = scenes.avatar_poses(wl["motion"], f)
        assert _run(nat, direct, poses) == 0
        sd = nat.dgsm_get_build_stats(direct.ctx)
        assert _run(nat, pers, poses) == 0
        sp = nat.dgsm_get_build_stats(pers.ctx)
        # the same binning: super-tile and tile pairs counted alike
        assert sp["n_pairs"] == sd["n_pairs"] > 1000
        assert sp["n_super_pairs"] == sd["n_super_pairs"]
        # motion and centroids: the same arithmetic, bit for bit
        assert torch.equal(pers.q_means, direct.q_means)
        assert torch.equal(pers.av_quats, direct.av_quats)
        assert torch.equal(pers.centroids, direct.centroids)
        # the atlas and the colours: the same sums in another order
        assert float(pers.dyn_atlas.min()) < 0.5
        assert torch.allclose(pers.dyn_atlas, direct.dyn_atlas, atol=1e-6, rtol=0)
        assert torch.allclose(pers.colors_out, direct.colors_out, atol=1e-5, rtol=1e-5)


def test_persistent_dynamic_atlas_matches_oracle(nat, orc, pair):
    wl, _, pers = pair
    poses = scenes.avatar_poses(wl["motion"], 61)
    assert _run(nat, pers, poses) == 0
    av = wl["avatars"]
    mr, qr = motion.rigid_transform(av.means, av.quats, wl["seg"], poses)
    moved = scenes.Scene(np.float32(mr), av.scales, np.float32(qr), av.opac, av.colors)
    lij = texel_sample(np.random.default_rng(31), 4, pers.H_dyn, pers.W_dyn, 24)
    tau = orc.build_tau_texels(moved, wl["lights"], pers.H_dyn, pers.W_dyn, wl["radii_dyn"], lij)
    got = pers.dyn_atlas.double().cpu().numpy()[lij[:, 0], :, lij[:, 1], lij[:, 2]]
    assert np.abs(got - np.exp(-tau)).max() <= 1e-4
    cen = motion.segment_centroids(pers.av_means.cpu().numpy(), av.opac, wl["seg"])
    assert np.abs(pers.centroids.cpu().numpy() - cen).max() <= 1e-6


def test_barrier_timeout_is_reported_and_the_context_builds_again(nat, pair):
    wl, direct, pers = pair
    poses = scenes.avatar_poses(wl["motion"], 51)
    assert _run(nat, direct, poses) == 0
    try:
        for b in (1, 2, 4, 6, 7):
            pers.timeout_barrier = b
            assert _run(nat, pers, poses) == DGSM_ERR_TIMEOUT, b
            pers.timeout_barrier = -1
            assert _run(nat, pers, poses) == 0
            assert torch.allclose(pers.dyn_atlas, direct.dyn_atlas, atol=1e-6, rtol=0)
            assert torch.allclose(pers.colors_out, direct.colors_out, atol=1e-5, rtol=1e-5)
    finally:
        pers.timeout_barrier = -1
    # an ordinary build on the same context after the aborted frames
    atl = nat.dgsm_build(pers.av_means, pers.av_scales, pers.av_quats, pers.av_opac, pers.lights, pers.H_dyn,
                         pers.W_dyn, pers.radii_dyn, params=dict(tile=8), ctx=pers.ctx, stream=pers.stream)
    pers.stream.synchronize()
    assert nat.dgsm_sync_status(pers.ctx) == 0
    assert torch.allclose(atl, direct.dyn_atlas, atol=1e-6, rtol=0)


def test_persistent_frame_over_capacity_is_reported_and_unshadowed(nat, pair):
    wl, direct, pers = pair
    poses = scenes.avatar_poses(wl["motion"], 12)
    assert _run(nat, pers, poses, max_pairs=1000) == DGSM_ERR_WORKSPACE
    assert bool((pers.dyn_atlas == 1.0).all())
    assert _run(nat, pers, poses) == 0
    assert _run(nat, direct, poses) == 0
    assert torch.allclose(pers.dyn_atlas, direct.dyn_atlas, atol=1e-6, rtol=0)


def test_persistent_frame_replays_in_a_graph(nat, pair):
    wl, _, pers = pair
    nodes = pers.capture()
    assert nodes <= 4  # pose copy, control memset, (tile cones,) the cooperative kernel
    for f in (5, 90):
        poses = scenes.avatar_poses(wl["motion"], f)
        pers.step_graph(poses)
        pers.stream.synchronize()
        assert nat.dgsm_sync_status(pers.ctx) == 0
        g_out, g_atl, g_means = pers.colors_out.clone(), pers.dyn_atlas.clone(), pers.q_means.clone()
        assert _run(nat, pers, poses) == 0
        assert torch.equal(pers.q_means, g_means)
        assert torch.allclose(pers.dyn_atlas, g_atl, atol=1e-6, rtol=0)
        assert torch.allclose(pers.colors_out, g_out, atol=1e-5, rtol=1e-5)
    for g in pers.graphs:
        g.close()
    pers.graphs = None


def _direct_frame(nat, st, av, seg, poses, lights, radii, Hs, Ws, Hd, Wd, radii_d, sh, static_atlas, max_pairs):
    """The frame by the separate library calls (the reference for the edge cases)."""
    L = lights.shape[0]
    mr, qr = (torch.empty((0, 3), device="cuda"), torch.empty((0, 4), device="cuda"))
    if av.n:
        mr, qr = nat.dgsm_rigid_transform(dev(av.means), dev(av.quats), seg, dev(poses))
    dyn = torch.ones((L, radii_d.shape[0], Hd, Wd), dtype=torch.float32, device="cuda")
    if av.n:
        nat.dgsm_build(mr, dev(av.scales), qr, dev(av.opac), lights, Hd, Wd, radii_d,
                       params=dict(tile=8, max_pairs=max_pairs), out=dyn)
    q = torch.cat([dev(st.means), mr]) if st.n else mr
    cin = dev(np.concatenate([st.colors, av.colors])) if st.n + av.n else torch.empty((0, 3), device="cuda")
    out = nat.dgsm_attenuate_dyn(static_atlas, radii, dyn, radii_d, lights, q, cin)
    cen = torch.zeros((len(seg) - 1, 3), dtype=torch.float32, device="cuda")
    if av.n:
        cen = nat.dgsm_segment_centroids(mr, dev(av.opac), seg)
        av_out = out[st.n:]
        nat.sh_relight_objects(sh, mr, qr, dev(av.scales), av_out, cen, seg, out=av_out)
    torch.cuda.synchronize()
    return dyn, out, cen


@pytest.mark.parametrize("n_static,n_each", [(0, [700, 313]), (900, []), (517, [0, 1, 457, 33])])
def test_persistent_frame_edge_cases(nat, n_static, n_each):
    """No avatars, no static receivers, and ragged objects (an empty one, a
    single Gaussian, sizes off every warp and block multiple): the persistent
    kernel gives the separate calls' frame."""
    rng = np.random.default_rng(7 + n_static)
    st = scenes.cube_scene(n_static, seed=61)
    av = scenes.cube_scene(int(sum(n_each)), seed=62, log_s_mean=np.log(0.05))
    seg = [0] + list(np.cumsum(n_each)) if n_each else [0, 0]
    n_obj = len(seg) - 1
    poses = np.zeros((n_obj, 8), np.float32)
    for o in range(n_obj):
        q = rng.normal(size=4)
        poses[o, :4] = q / np.linalg.norm(q)
        poses[o, 4:7] = rng.uniform(-0.3, 0.3, 3)
    lights = dev(np.float32([[0, 0, 0], [0.5, -0.4, 0.8]]))
    radii, radii_d = dev(scenes.radii_linear(0.1, 8, 12)), dev(scenes.radii_linear(0.1, 8, 10))
    Hs = Ws = 32
    Hd, Wd = 40, 24
    D, Y, w = scenes.cubemap_samples(16, seed=5)
    sh = nat.sh_fit(dev(D), dev(Y), dev(w))
    static_atlas = torch.ones((2, 12, Hs, Ws), dtype=torch.float32, device="cuda")
    if st.n:
        static_atlas = nat.dgsm_build(dev(st.means), dev(st.scales), dev(st.quats), dev(st.opac), lights, Hs, Ws,
                                      radii)
    max_pairs = 300000
    dyn_ref, out_ref, cen_ref = _direct_frame(nat, st, av, seg, poses, lights, radii, Hs, Ws, Hd, Wd, radii_d, sh,
                                              static_atlas, max_pairs)
    n = st.n + av.n
    q_means = dev(np.concatenate([st.means, av.means])) if n else torch.empty((0, 3), device="cuda")
    cin = dev(np.concatenate([st.colors, av.colors])) if n else torch.empty((0, 3), device="cuda")
    cout = torch.full_like(cin, -1.0)
    quats_out = torch.empty((av.n, 4), dtype=torch.float32, device="cuda")
    dyn = torch.full((2, 10, Hd, Wd), -1.0, dtype=torch.float32, device="cuda")
    cen = torch.full((n_obj, 3), -1.0, dtype=torch.float32, device="cuda")
    rest_m = dev(av.means) if av.n else torch.empty((0, 3), device="cuda")
    rest_q = dev(av.quats) if av.n else torch.empty((0, 4), device="cuda")
    scl = dev(av.scales) if av.n else torch.empty((0, 3), device="cuda")
    opc = dev(av.opac) if av.n else torch.empty((0,), device="cuda")
    nat.dgsm_crowd_frame(q_means, cin, cout, st.n, static_atlas, radii, rest_m, rest_q, scl, opc, quats_out, seg,
                         dev(poses), dyn, radii_d, lights, sh, cen, params=dict(max_pairs=max_pairs))
    torch.cuda.synchronize()
    assert nat.dgsm_sync_status() == 0
    assert torch.allclose(dyn, dyn_ref, atol=1e-6, rtol=0)
    assert torch.allclose(cout, out_ref, atol=1e-5, rtol=1e-5)
    assert torch.equal(cen, cen_ref)
