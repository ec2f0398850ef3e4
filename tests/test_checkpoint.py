"""Checkpoint files of the field's training state: round trip, shapes, and
rejection of damaged files (host only)."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import checkpoint


def test_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    p, m, v = (torch.tensor(rng.standard_normal((2, 1000)), dtype=torch.float32) for _ in range(3))
    mask = torch.tensor(rng.integers(0, 2, 4096), dtype=torch.uint8)
    f = str(tmp_path / "field.ckpt")
    checkpoint.save_field(f, p, m, v, step=1234, mask=mask)
    p2, m2, v2, step, mask2 = checkpoint.load_field(f)
    assert step == 1234
    assert torch.equal(p, p2) and torch.equal(m, m2) and torch.equal(v, v2) and torch.equal(mask, mask2)
    checkpoint.save_field(f, p[0], m[0], v[0], step=0)   # one light, no mask
    p3, _, _, step, mask3 = checkpoint.load_field(f)
    assert p3.shape == (1, 1000) and torch.equal(p3[0], p[0]) and step == 0 and mask3 is None


def test_damaged_files_are_rejected(tmp_path):
    f = str(tmp_path / "field.ckpt")
    z = torch.zeros(10)
    checkpoint.save_field(f, z, z, z, step=3)
    data = open(f, "rb").read()
    open(f, "wb").write(data[:-4])
    with pytest.raises(ValueError):
        checkpoint.load_field(f)
    open(f, "wb").write(b"NOTAFILE" + data[8:])
    with pytest.raises(ValueError):
        checkpoint.load_field(f)
    with pytest.raises(ValueError):
        checkpoint.save_field(f, z, torch.zeros(11), z, step=0)
