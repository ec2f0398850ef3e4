"""GPU parity of the receiver-driven region of interest (Sec. 3.2): the
region's texel mask and shell ranges bit-exact against the oracle's FP32
specification, the region's atlas against the FP64 oracle (dense values on
the region, 1 elsewhere), attenuation of the receivers in the box equal to
attenuation through the dense atlas, the avatar box, and the room workload of
the benchmark."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev, texel_sample

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _in_box(p, box):
    p = np.asarray(p, dtype=np.float32)
    return ((np.abs(p[:, 0] - box[0]) <= box[2]) & (np.abs(p[:, 1] - box[1]) <= box[2]) &
            (p[:, 2] >= box[3]) & (p[:, 2] <= box[4]))


@pytest.mark.parametrize("tile", [8, 16])
def test_roi_build_matches_oracle(nat, orc, tile):
    occ = scenes.cube_scene(1500, seed=0)
    recv = scenes.cube_scene(6000, seed=1)
    lights = np.float32([[0, 0, 0], [0.8, 0.5, 1.2]])
    radii = scenes.radii_geometric(0.2, 9.0, 12)
    H, W = 40, 56
    box = np.float32([0.3, -0.4, 1.1, 2.0, 4.2])
    d = scene_to_dev(occ)
    atlas, mask, kr = nat.dgsm_build_roi(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W,
                                         dev(radii), dev(recv.means), dev(box), params={"tile": tile},
                                         want_roi=True)
    omask, okr = orc.f32_roi(recv.means, box, lights, H, W, radii)
    assert np.array_equal(mask.cpu().numpy(), omask)
    assert np.array_equal(kr.cpu().numpy(), okr)
    ref = orc.roi_atlas(orc.build_atlas(occ, lights, H, W, radii), omask, okr)
    got = atlas.double().cpu().numpy()
    assert np.abs(got - ref).max() <= TOL
    assert (got[ref == 1.0] == 1.0).all()  # outside the region exactly 1
    # receivers in the box see the dense atlas
    dense = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii),
                           params={"tile": tile})
    sel = _in_box(recv.means, box)
    c_r, T_r = nat.dgsm_attenuate(atlas, dev(radii), dev(lights), dev(recv.means[sel]), dev(recv.colors[sel]),
                                  want_T=True)
    c_d, T_d = nat.dgsm_attenuate(dense, dev(radii), dev(lights), dev(recv.means[sel]), dev(recv.colors[sel]),
                                  want_T=True)
    assert (T_r - T_d).abs().max().item() <= 1e-6
    assert T_d.min().item() < 0.9


def test_roi_box_matches_oracle(nat, orc):
    av = scenes.avatar_body(np.random.default_rng(4), 20000)
    box = nat.dgsm_roi_box(dev(av.means), dev(av.opac), R=2.0, z_margin=0.1).cpu().numpy()
    ref = orc.roi_box(av.means, av.opac, R=2.0, z_margin=0.1)
    assert np.abs(box - ref).max() <= 1e-5


def test_roi_edge_cases(nat):
    occ = scenes.cube_scene(500, seed=2)
    lights = np.float32([[0, 0, 0]])
    radii = scenes.radii_linear(0.1, 8, 8)
    d = scene_to_dev(occ)
    none = dev(np.zeros((0, 3), np.float32))
    atlas, mask, kr = nat.dgsm_build_roi(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 16, 16,
                                         dev(radii), none, dev([0, 0, 1, 0, 1]), want_roi=True)
    assert (atlas == 1).all() and mask.sum().item() == 0 and kr.tolist() == [[8, -1]]
    recv = dev(scenes.cube_scene(100, seed=3).means)
    atlas = nat.dgsm_build_roi(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 16, 16,
                               dev(radii), recv, dev([0, 0, -1, 0, 1]))  # R < 0: empty box
    assert (atlas == 1).all()


def test_room_roi_build(nat, orc):
    """The benchmark's room: box around the avatar, all 1.6M Gaussians as
    receivers; the region against the dense build and sampled oracle texels."""
    wl = scenes.workload("room1p6m")
    sc = wl["occluders"]
    sl = sc.meta["avatar"]
    d = scene_to_dev(sc)
    lights, radii = dev(wl["lights"]), dev(wl["radii"])
    H, W = wl["H"], wl["W"]
    box = np.float32(orc.roi_box(sc.means[sl], sc.opac[sl], R=2.0, z_margin=0.1))
    atlas, mask, kr = nat.dgsm_build_roi(d["means"], d["scales"], d["quats"], d["opac"], lights, H, W, radii,
                                         d["means"], dev(box), want_roi=True)
    omask, okr = orc.f32_roi(sc.means, box, wl["lights"], H, W, wl["radii"])
    assert np.array_equal(mask.cpu().numpy(), omask) and np.array_equal(kr.cpu().numpy(), okr)
    assert 0.01 < omask.mean() < 0.7
    dense = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, H, W, radii)
    g, dn = atlas.cpu().numpy(), dense.cpu().numpy()
    k0, k1 = okr[0]
    sel = omask[0].astype(bool)
    assert np.abs(g[0, k0:k1 + 1][:, sel] - dn[0, k0:k1 + 1][:, sel]).max() <= 1e-6
    rest = np.ones_like(g, dtype=bool)
    rest[0, k0:k1 + 1][:, sel] = False
    assert (g[rest] == 1.0).all()
    # sampled texels of the region against the FP64 oracle
    ii, jj = np.nonzero(omask[0])
    pick = np.random.default_rng(5).choice(ii.size, 12, replace=False)
    lij = np.stack([np.zeros(12, np.int32), ii[pick], jj[pick]], 1).astype(np.int32)
    tau = orc.build_tau_texels(sc, wl["lights"], H, W, wl["radii"], lij)
    ref = np.exp(-tau)[:, k0:k1 + 1]
    assert np.abs(g[0, k0:k1 + 1][:, ii[pick], jj[pick]].T - ref).max() <= TOL
