"""Resuming the field's training from a checkpoint: 40 Adam steps, a save
and load through the file, 40 more steps from step0 = 40, against 80 steps
in one run (the voxel draws and the bias correction depend only on the seed
and the step number)."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import checkpoint, scenes

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def test_resume_matches_one_run(nat, tmp_path):
    sc = scenes.cube_scene(2000, seed=0)
    d = scene_to_dev(sc)
    radii = scenes.radii_linear(0.1, 8, 16)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 64, 64, dev(radii))[0]
    p0 = nat.nf_init(seed=3)
    pa, ma, va = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    la = nat.nf_train(atlas, pa, ma, va, 80, batch=4096, seed=9)
    pb, mb, vb = p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)
    lb1 = nat.nf_train(atlas, pb, mb, vb, 40, batch=4096, seed=9)
    f = str(tmp_path / "field.ckpt")
    checkpoint.save_field(f, pb, mb, vb, step=40)
    pc, mc, vc, step, _ = checkpoint.load_field(f, device="cuda")
    pc, mc, vc = pc[0].contiguous(), mc[0].contiguous(), vc[0].contiguous()
    lb2 = nat.nf_train(atlas, pc, mc, vc, 40, batch=4096, seed=9, step0=step)
    lb = torch.cat([lb1, lb2])
    assert torch.allclose(lb, la, rtol=1e-4, atol=1e-7)
    scale = pa.abs().max().item()
    assert (pc - pa).abs().max().item() <= 1e-4 * scale
    assert la[-10:].mean() < la[:10].mean()  # it trains
