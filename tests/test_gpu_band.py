"""GPU parity of the row-band split of one light set's atlas (the multi-GPU
path when there are fewer lights than GPUs): every band built on its own
(dgsm_build_band) and put back with dgsm_atlas_rows_copy, as the ranks of
shard.banded_atlas do after their all-gather, equals the dense build; a band
alone against the FP64 oracle; T = 1 outside the band; argument checks.

A band's tiles get the same pair lists as in the dense build, so only the
order of the shared-memory float additions inside a tile differs between
the two: 1e-6.  Against the oracle the build's own bound, 1e-4."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes, shard

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _banded(nat, d, lights, H, W, radii, world, params=None):
    p = dict(params or {})
    tile = int(p.get("tile", 8))
    dt = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[int(p.get("atlas_dtype", 0))]
    L, K = lights.shape[0], radii.shape[0]
    atlas = torch.empty((L, K, H, W), dtype=dt, device="cuda")
    for r in range(world):            # the ranks, one after the other on this GPU
        r0, r1, hb = shard.band_rows(H, tile, r, world)
        if r1 == r0:
            continue
        full = nat.dgsm_build_band(d["means"], d["scales"], d["quats"], d["opac"], lights, H, W, radii, r0, r1,
                                   params=params)
        out = full.cpu()
        assert (out[:, :, :r0] == 1).all() and (out[:, :, r1:] == 1).all()
        slab = torch.empty((L, K, hb, W), dtype=dt, device="cuda")
        nat.dgsm_atlas_rows_copy(full, r0, slab, 0, r1 - r0)
        nat.dgsm_atlas_rows_copy(slab, 0, atlas, r0, r1 - r0)
    return atlas


@pytest.mark.parametrize("world,tile", [(2, 8), (3, 8), (8, 8), (5, 16)])
def test_bands_reassemble_the_dense_build(nat, world, tile):
    sc = scenes.cube_scene(20000, seed=0)
    d = scene_to_dev(sc)
    lights = dev(scenes.four_lights())
    radii = dev(scenes.radii_linear(0.1, 8, 16))
    H, W = 72, 64
    dense = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, H, W, radii,
                           params={"tile": tile})
    got = _banded(nat, d, lights, H, W, radii, world, params={"tile": tile})
    assert (got - dense).abs().max().item() <= 1e-6
    assert dense.min().item() < 0.5


def test_cube_map_bands(nat):
    """The split works the same on a cube-map atlas (six 24 x 24 faces)."""
    sc = scenes.cube_scene(8000, seed=6)
    d = scene_to_dev(sc)
    lights = dev(scenes.four_lights()[:2])
    radii = dev(scenes.radii_linear(0.1, 8, 8))
    p = {"atlas_map": 1}
    dense = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, 144, 24, radii, params=p)
    got = _banded(nat, d, lights, 144, 24, radii, 4, params=p)
    assert (got - dense).abs().max().item() <= 1e-6


def test_band_against_the_oracle(nat, orc):
    sc = scenes.cube_scene(1500, seed=2)
    lights = np.float32([[0, 0, 0], [0.5, -0.5, 1.0]])
    radii = scenes.radii_linear(0.1, 8, 8)
    H, W = 40, 24
    d = scene_to_dev(sc)
    band = nat.dgsm_build_band(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii),
                               16, 32).double().cpu().numpy()
    ref = orc.build_atlas(sc, lights, H, W, radii)
    assert np.abs(band[:, :, 16:32] - ref[:, :, 16:32]).max() <= 1e-4
    assert (band[:, :, :16] == 1).all() and (band[:, :, 32:] == 1).all()


def test_room_split_over_eight(nat):
    """The benchmark's room atlas (512 x 512 x 64, 1.6M Gaussians) in eight
    bands of 64 rows against the dense build."""
    wl = scenes.workload("room1p6m")
    d = scene_to_dev(wl["occluders"])
    lights, radii = dev(wl["lights"]), dev(wl["radii"])
    dense = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, 512, 512, radii)
    got = _banded(nat, d, lights, 512, 512, radii, 8)
    assert (got - dense).abs().max().item() <= 1e-6


def test_half_precision_rows_and_one_rank(nat):
    sc = scenes.cube_scene(3000, seed=4)
    d = scene_to_dev(sc)
    lights = dev(scenes.four_lights())
    radii = dev(scenes.radii_linear(0.1, 8, 8))
    p = {"atlas_dtype": 2}
    dense = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, 48, 40, radii, params=p)
    got = _banded(nat, d, lights, 48, 40, radii, 3, params=p)
    assert (got.float() - dense.float()).abs().max().item() <= 2 ** -8
    one = shard.build_banded(nat, d["means"], d["scales"], d["quats"], d["opac"], lights, 48, 40, radii, params=p)
    assert (one.float() - dense.float()).abs().max().item() <= 2 ** -8


def test_bad_bands_are_refused(nat):
    from paper_2601_01660_b300._native import DGSMError
    sc = scenes.cube_scene(10, seed=1)
    d = scene_to_dev(sc)
    radii = dev(scenes.radii_linear(0.1, 8, 4))
    for r0, r1 in [(8, 8), (-8, 8), (0, 40), (16, 8)]:
        with pytest.raises(DGSMError):
            nat.dgsm_build_band(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 32, 32, radii,
                                r0, r1)
    a = torch.ones((1, 4, 32, 32), device="cuda")
    b = torch.ones((1, 4, 8, 32), device="cuda")
    with pytest.raises(DGSMError):
        nat.dgsm_atlas_rows_copy(a, 28, b, 0, 8)      # past the end of the source
    with pytest.raises(DGSMError):
        nat.dgsm_atlas_rows_copy(a, 0, b, 4, 8)       # past the end of the slab
