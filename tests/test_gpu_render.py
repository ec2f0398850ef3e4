"""GPU parity of the splat renderer: the cubemap probe (Sec. 3.4) and pinhole
cameras (the final composite) against the brute-force oracle (every Gaussian
at every pixel), the pixel directions and solid angles, the probe of the
benchmark's room fed to the SH fit, and a 320 x 240 view of the room.

Tolerance: the inclusion test (Mahalanobis distance <= 3) and the depth order
are the same single-precision operations on both sides, so the same splats
reach a pixel in the same order.  alpha uses the kernel's exp in FP32 against
FP64 in the oracle (relative 1e-6), the kernel composites in FP32 over a few
hundred splats per pixel, and it leaves out what lies behind a transmittance
below 1e-6 (at most 1e-6 of a colour in [0, 1]).  Bound: 2e-5 per channel."""
import numpy as np
import pytest
import torch
from scipy import integrate

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _render(nat, sc, centre, face, near=0.05):
    d = scene_to_dev(sc)
    return nat.dgsm_render_cubemap(d["means"], d["scales"], d["quats"], d["opac"], d["colors"], dev(centre),
                                   face=face, near=near, want_pairs=True)


@pytest.mark.parametrize("face", [8, 16, 24])
def test_render_matches_oracle_every_pixel(nat, orc, face):
    sc = scenes.cube_scene(3000, seed=face, centre=(0.0, 0.0, 0.0), side=6.0)
    centre = np.float32([0.1, -0.2, 0.3])
    rgb, P = _render(nat, sc, centre, face)
    ref = orc.render_pixels(sc, centre, face, np.arange(6 * face * face))
    err = np.abs(rgb.double().cpu().numpy() - ref)
    assert P > 0 and ref.max() > 0.3
    assert err.max() <= TOL and np.median(err) <= 1e-6, err.max()


def test_render_large_splats_and_near_plane(nat, orc):
    # Gaussians close to the probe cover many tiles and straddle faces
    rng = np.random.default_rng(3)
    sc = scenes.cube_scene(400, seed=4, centre=(0.0, 0.0, 0.0), side=1.0, log_s_mean=np.log(0.1))
    sc.means[:20] = np.float32(rng.uniform(-0.06, 0.06, (20, 3)))  # some behind the near plane
    rgb, _ = _render(nat, sc, [0, 0, 0], 16, near=0.05)
    ref = orc.render_pixels(sc, [0, 0, 0], 16, np.arange(6 * 256), near=0.05)
    assert np.abs(rgb.double().cpu().numpy() - ref).max() <= TOL


def test_render_empty(nat):
    sc = scenes.cube_scene(1, seed=0)
    d = scene_to_dev(scenes.subset(sc, np.arange(0)))
    rgb = nat.dgsm_render_cubemap(d["means"], d["scales"], d["quats"], d["opac"], d["colors"], dev([0, 0, 0]),
                                  face=8)
    assert rgb.shape == (384, 3) and (rgb == 0).all()
    from paper_2601_01660_b300._native import DGSMError
    with pytest.raises(DGSMError):
        nat.dgsm_render_cubemap(d["means"], d["scales"], d["quats"], d["opac"], d["colors"], dev([0, 0, 0]),
                                face=12)


def test_render_nothing_in_view(nat):
    """Gaussians that no camera sees (all behind it, or transparent): no
    splat reaches a tile and the image stays black."""
    sc = scenes.cube_scene(500, seed=9, centre=(0.0, 0.0, 3.0), side=2.0)
    sc.opac[:100] = 0.0
    d = scene_to_dev(sc)
    cam = scenes.look_at_camera([0, 0, 0], [1.0, 0, 0], 32, 24, 60.0)   # the cube is 63 degrees above the view axis
    rgb, P = nat.dgsm_render_views(d["means"], d["scales"], d["quats"], d["opac"], d["colors"], dev(cam[None]),
                                   32, 24, want_pairs=True)
    assert P == 0 and (rgb == 0).all()


def test_cube_dirs_and_solid_angles(nat, orc):
    face = 16
    dirs, w = nat.dgsm_cube_dirs(face)
    dirs, w = dirs.cpu().numpy(), w.double().cpu().numpy()
    assert np.abs(dirs - orc.cube_dirs(face)).max() <= 1e-6
    assert abs(w.sum() - 4 * np.pi) <= 1e-5
    for p in (0, 37, 255, 256 * 3 + 100):
        i, j = (p % 256) // face, p % face
        u0, v0 = 2 * j / face - 1, 2 * i / face - 1
        ref, _ = integrate.dblquad(lambda v, u: (1 + u * u + v * v) ** -1.5, u0, u0 + 2 / face, v0, v0 + 2 / face)
        assert abs(w[p] - ref) <= 1e-7 * max(1.0, ref / 1e-3)


def test_room_probe_sampled_pixels_and_fit(nat, orc):
    """The benchmark's room without its avatar, probed at the avatar's
    alpha-weighted centroid: 300 sampled pixels against the oracle, then the
    SH fit of the rendered probe against the FP64 oracle fit."""
    wl = scenes.workload("room1p6m")
    sc = wl["occluders"]
    sl = sc.meta["avatar"]
    keep = np.concatenate([np.arange(0, sl.start), np.arange(sl.stop, sc.n)])
    scene = scenes.subset(sc, keep)
    av = scenes.subset(sc, np.arange(sl.start, sl.stop))
    cen = nat.dgsm_weighted_centroid(dev(av.means), dev(av.opac))
    centre = cen.cpu().numpy().astype(np.float32)
    face = 64
    rgb, P = _render(nat, scene, centre, face)
    pix = np.random.default_rng(7).choice(6 * face * face, 300, replace=False)
    ref = orc.render_pixels(scene, centre, face, pix)
    got = rgb.double().cpu().numpy()[pix]
    assert np.abs(got - ref).max() <= TOL
    assert np.median(ref.sum(1)) > 0.1  # the room is around the probe
    dirs, w = nat.dgsm_cube_dirs(face)
    sh, sh64 = nat.sh_fit(dirs, rgb, w, want64=True)
    sh_ref = orc.sh_fit(dirs.cpu().numpy(), rgb.cpu().numpy(), w.cpu().numpy())
    assert np.allclose(sh64.cpu().numpy(), sh_ref, rtol=1e-9, atol=1e-12)


def test_render_views_matches_oracle_every_pixel(nat, orc):
    sc = scenes.cube_scene(3000, seed=11, centre=(0.0, 0.0, 0.0), side=6.0)
    W, H = 40, 28   # not multiples of the 8-pixel tile
    cams = np.stack([scenes.look_at_camera([0.2, -2.5, 0.4], [0, 0, 0], W, H, 70.0),
                     scenes.look_at_camera([1.5, 1.0, -0.5], [0.1, 0.2, 0.3], W, H, 45.0)])
    d = scene_to_dev(sc)
    rgb, P = nat.dgsm_render_views(d["means"], d["scales"], d["quats"], d["opac"], d["colors"], dev(cams), W, H,
                                   want_pairs=True)
    ref = orc.render_view_pixels(sc, cams, W, H, np.arange(2 * W * H))
    err = np.abs(rgb.double().cpu().numpy().reshape(-1, 3) - ref)
    assert P > 0 and ref.max() > 0.3
    assert err.max() <= TOL and np.median(err) <= 1e-6, err.max()


def test_room_composite_sampled_pixels(nat, orc):
    """The final composite: the room with its avatar seen from 3 m, 320 x 240,
    on 300 sampled pixels (the scene's own colours; the renderer alone)."""
    wl = scenes.workload("room1p6m")
    sc = wl["occluders"]
    cam = scenes.look_at_camera([-1.2, -1.5, 1.6], [1.5, 0.0, 0.9], 320, 240, 60.0)
    d = scene_to_dev(sc)
    rgb = nat.dgsm_render_views(d["means"], d["scales"], d["quats"], d["opac"], d["colors"], dev(cam[None]),
                                320, 240)
    pix = np.random.default_rng(8).choice(320 * 240, 300, replace=False)
    ref = orc.render_view_pixels(sc, cam[None], 320, 240, pix)
    assert np.abs(rgb.double().cpu().numpy().reshape(-1, 3)[pix] - ref).max() <= TOL
    assert np.median(ref.sum(1)) > 0.1
