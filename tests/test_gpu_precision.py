"""Storage precision on the 3M-Gaussian, 4-light cube workload (64x64x16):
float32, float16 and bfloat16 atlases (tau accumulated in float32 for all
three) against the FP64 oracle on a random texel sample, per light."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev, texel_sample

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f16": 2e-3, "bf16": 2.0 ** -9 + 1e-4}


def test_precision_per_light_against_oracle(orc):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    nat = native()
    wl = scenes.workload("cube3m4l")
    sc, lights, radii, H, W = wl["occluders"], wl["lights"], wl["radii"], wl["H"], wl["W"]
    d = scene_to_dev(sc)
    lij = texel_sample(np.random.default_rng(4), lights.shape[0], H, W, 128)
    ref = np.exp(-orc.build_tau_texels(sc, lights, H, W, radii, lij))
    table = {}
    for dt, tol in TOL.items():
        a = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W,
                           dev(radii), params=dict(atlas_dtype=dt))
        got = a.double().cpu().numpy()[lij[:, 0], :, lij[:, 1], lij[:, 2]]
        err = np.abs(got - ref)
        table[dt] = {f"light{l}": {"max": float(err[lij[:, 0] == l].max()),
                                   "mean": float(err[lij[:, 0] == l].mean())}
                     for l in range(lights.shape[0])}
        assert err.max() <= tol, (dt, err.max())
    path = os.environ.get("DGSM_REPORT_DIR")
    if path:
        with open(os.path.join(path, "precision_vs_oracle.json"), "w") as f:
            json.dump({"workload": "cube3m4l", "sample": "128 texels x 16 shells", "abs_dT": table}, f)
