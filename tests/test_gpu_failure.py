"""Failure detection without a GPU fault: a bounded device-side wait that
nothing completes gives up, records DGSM_ERR_TIMEOUT in the status word and
returns; the host reads the status and the context stays usable.  Input
faults are reported through the same word (non-finite Gaussians) or as
argument errors before any launch."""
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


def test_bounded_wait_completes_and_times_out(nat):
    assert nat.dgsm_sync_status() == nat.DGSM_OK
    nat.dgsm_selftest_wait(arrive=True, limit=4096)
    assert nat.dgsm_sync_status() == nat.DGSM_OK
    nat.dgsm_selftest_wait(arrive=False, limit=4096)     # nothing arrives
    assert nat.dgsm_sync_status() == 4                   # DGSM_ERR_TIMEOUT, then cleared
    assert nat.dgsm_sync_status() == nat.DGSM_OK
    # the context and the device still work
    sc = scenes.cube_scene(500, seed=1)
    d = scene_to_dev(sc)
    radii = scenes.radii_linear(0.1, 8, 8)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev([[0, 0, 0]]), 16, 16, dev(radii))
    torch.cuda.synchronize()
    assert torch.isfinite(atlas).all() and nat.dgsm_sync_status() == nat.DGSM_OK
    with pytest.raises(nat.DGSMError):
        nat.dgsm_selftest_wait(arrive=False, limit=0)
