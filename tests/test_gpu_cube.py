"""GPU parity of the cube-map atlas (ablation (C) of Sec. 4): the build
against the FP64 oracle, the binning bit-exact against the oracle's FP32
specification (faces of one to six tiles), the
lookup's integer decisions bit-exact, the attenuation through a cube atlas
against the oracle, the receiver region, and the shape checks.

Tolerances are those of the octahedral paths: the build 1e-4 (FP32 Eq. 3
over a few hundred Gaussians per texel against FP64), the attenuation 1e-5
(an FP32 trilinear blend of the same atlas values)."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu

CUBE = {"atlas_map": 1}


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _scene():
    rng = np.random.default_rng(5)
    flat = scenes.cube_scene(500, seed=41, log_s_mean=np.log(0.12))
    flat.scales[np.arange(flat.n), rng.integers(0, 3, flat.n)] = 0.002
    return scenes.concat(scenes.cube_scene(1500, seed=2), flat)


@pytest.mark.parametrize("F,tile", [(8, 8), (24, 8), (16, 16), (40, 8)])
def test_build_and_binning(nat, orc, F, tile):
    sc = _scene()
    lights = np.float32([[0, 0, 0], [0.5, -0.5, 1.0]])
    radii = scenes.radii_linear(0.1, 8, 8)
    H = 6 * F
    d = scene_to_dev(sc)
    p = dict(CUBE, tile=tile)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, F, dev(radii),
                           params=p)
    with orc.atlas_map(1):
        ref = orc.build_atlas(sc, lights, H, F, radii)
        ko, vo = orc.f32_bin(sc, lights, H, F, radii, tile=tile)
    assert np.abs(atlas.double().cpu().numpy() - ref).max() <= 1e-4
    assert ref.min() < 0.9
    kg, vg = nat.dgsm_bin(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, F, dev(radii),
                          params=p)
    assert np.array_equal(kg.cpu().numpy().view(np.uint32), ko)
    assert np.array_equal(vg.cpu().numpy().view(np.uint32), vo)


def test_sample_index_bit_exact(nat, orc):
    rng = np.random.default_rng(3)
    F = 64
    radii = scenes.radii_geometric(0.05, 12, 33)
    o = np.float32([0.3, -0.2, 1.0])
    pts = np.float32(rng.uniform(-6, 6, (4000, 3)))
    pts[:50] = o                                            # at the light
    pts[50:100] = o + np.float32(rng.choice([-1, 1], (50, 1))) * np.float32([[1, 1, 0]])   # |x| = |y| ties
    pts[100:150] = o + np.float32([[0, 2, -2]]) * np.float32(rng.uniform(0.1, 3, (50, 1)))  # |y| = |z| ties
    pts[150:200] = o + radii[rng.integers(0, 33, 50)][:, None] * np.float32([0, 0, 1])     # on shells
    with orc.atlas_map(1):
        oi, of = orc.f32_sample_index(pts, o, 6 * F, F, radii)
    gi, gf = nat.dgsm_sample_index_cube(dev(pts), dev(o), F, dev(radii))
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(gf.cpu().numpy().view(np.uint32), of.view(np.uint32))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_attenuate_matches_oracle(nat, orc, dtype):
    rng = np.random.default_rng(9)
    L, K, F = 3, 6, 24
    radii = scenes.radii_geometric(0.2, 9.0, K)
    atlas = dev(rng.random((L, K, 6 * F, F)), dtype)
    lights = np.float32(rng.normal(0, 1, (L, 3)))
    q = scenes.cube_scene(5000, seed=12)
    qm = q.means.copy()
    qm[:20] = lights[0]                                     # receivers at a light
    lw = np.float32([0.5, 0.3, 0.2])
    out, T = nat.dgsm_attenuate_cube(atlas, dev(radii), dev(lights), dev(qm), dev(q.colors), light_w=dev(lw),
                                     direct_frac=0.8, want_T=True)
    with orc.atlas_map(1):
        ref, Tref = orc.attenuate(atlas.double().cpu().numpy(), radii, lights, qm, q.colors, light_w=lw,
                                  direct_frac=0.8, want_T=True)
    assert np.abs(T.double().cpu().numpy() - Tref).max() <= 1e-5
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 1e-5
    assert (T[:20, 0] == 1).all()


def test_build_then_attenuate(nat, orc):
    sc = _scene()
    lights = np.float32([[0, 0, 0]])
    radii = scenes.radii_linear(0.1, 8, 8)
    F = 16
    d = scene_to_dev(sc)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 6 * F, F, dev(radii),
                           params=CUBE)
    out, T = nat.dgsm_attenuate_cube(atlas, dev(radii), dev(lights), d["means"], d["colors"], want_T=True)
    with orc.atlas_map(1):
        ref, Tref = orc.attenuate(atlas.double().cpu().numpy(), radii, lights, sc.means, sc.colors, want_T=True)
    assert np.abs(T.double().cpu().numpy() - Tref).max() <= 1e-5
    assert Tref.min() < 0.5


def test_roi_build(nat, orc):
    occ = scenes.cube_scene(400, seed=0)
    recv = scenes.cube_scene(3000, seed=1)
    lights = np.float32([[0, 0, 0], [0.8, 0.5, 1.2]])
    radii = scenes.radii_geometric(0.2, 9.0, 10)
    box = np.float32([0.3, -0.4, 1.1, 2.0, 4.2])
    F = 16
    d = scene_to_dev(occ)
    atlas, mask, kr = nat.dgsm_build_roi(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 6 * F, F,
                                         dev(radii), dev(recv.means), dev(box), params=dict(CUBE, tile=8),
                                         want_roi=True)
    with orc.atlas_map(1):
        omask, okr = orc.f32_roi(recv.means, box, lights, 6 * F, F, radii)
        ref = orc.roi_atlas(orc.build_atlas(occ, lights, 6 * F, F, radii), omask, okr)
    assert np.array_equal(mask.cpu().numpy(), omask)
    assert np.array_equal(kr.cpu().numpy(), okr)
    assert np.abs(atlas.double().cpu().numpy() - ref).max() <= 1e-4


def test_shapes_are_checked(nat):
    sc = scenes.cube_scene(10, seed=1)
    d = scene_to_dev(sc)
    from paper_2601_01660_b300._native import DGSMError
    radii = dev(scenes.radii_linear(0.1, 8, 4))
    with pytest.raises(DGSMError):   # a cube atlas has H = 6 W
        nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 40, 8, radii,
                       params=CUBE)
    with pytest.raises(DGSMError):   # the face must be a whole number of tiles
        nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 72, 12, radii,
                       params=dict(CUBE, tile=8))
    with pytest.raises(DGSMError):   # no such parameterisation
        nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 48, 8, radii,
                       params={"atlas_map": 2})
    with pytest.raises(ValueError):
        nat.dgsm_attenuate_cube(torch.ones(1, 4, 40, 8, device="cuda"), radii, dev([[0, 0, 0]]),
                                d["means"], d["colors"])
