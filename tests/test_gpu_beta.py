"""GPU parity of the opacity-to-absorption mappings (ablation (B) of Sec. 4):
the build against the FP64 oracle under each mapping, and the binning (whose
culling radius depends on the mapping) bit-exact against the oracle's FP32
specification."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_build_and_binning_per_mapping(nat, orc, mode):
    rng = np.random.default_rng(mode)
    flat = scenes.cube_scene(600, seed=40 + mode, log_s_mean=np.log(0.1))
    flat.scales[np.arange(flat.n), rng.integers(0, 3, flat.n)] = 0.002   # 2 mm thick discs
    sc = scenes.concat(scenes.cube_scene(1500, seed=0), flat)
    lights = np.float32([[0, 0, 0], [0.5, -0.5, 1.0]])
    radii = scenes.radii_linear(0.1, 8, 8)
    H, W = 24, 40
    d = scene_to_dev(sc)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii),
                           params={"beta_mode": mode})
    with orc.beta_mode(mode):
        ref = orc.build_atlas(sc, lights, H, W, radii)
        ko, vo = orc.f32_bin(sc, lights, H, W, radii)
    assert np.abs(atlas.double().cpu().numpy() - ref).max() <= 1e-4
    assert ref.min() < 0.9
    kg, vg = nat.dgsm_bin(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii),
                          params={"beta_mode": mode})
    assert np.array_equal(kg.cpu().numpy().view(np.uint32), ko)
    assert np.array_equal(vg.cpu().numpy().view(np.uint32), vo)


def test_bad_beta_mode_is_rejected(nat):
    sc = scenes.cube_scene(10, seed=1)
    d = scene_to_dev(sc)
    from paper_2601_01660_b300._native import DGSMError
    for mode in (0, 5):
        with pytest.raises(DGSMError):
            nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 8, 8,
                           dev(scenes.radii_linear(0.1, 8, 4)), params={"beta_mode": mode})
