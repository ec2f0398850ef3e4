"""Pins of the receiver-driven region of interest (Sec. 3.2, "Receiver-driven
ROI"): the region covers every voxel a receiver in the box reads (attenuation
through the region's atlas equals attenuation through the dense atlas), every
marked texel is read by one of them (a numpy restatement from the FP32 index
specification), the box of an avatar in closed form, and the empty cases."""
import numpy as np

import oracle
from paper_2601_01660_b300 import scenes


def _setup(seed=0, H=24, W=32, K=10):
    occ = scenes.cube_scene(400, seed=seed)
    recv = scenes.cube_scene(3000, seed=seed + 1)
    lights = np.float32([[0, 0, 0], [0.8, 0.5, 1.2]])
    radii = scenes.radii_geometric(0.2, 9.0, K)
    box = np.float32([0.3, -0.4, 1.1, 2.0, 4.2])
    return occ, recv, lights, radii, box, H, W


def _in_box(p, box):
    p = np.asarray(p, dtype=np.float32)
    dx = np.abs(p[:, 0] - box[0])
    dy = np.abs(p[:, 1] - box[1])
    return (dx <= box[2]) & (dy <= box[2]) & (p[:, 2] >= box[3]) & (p[:, 2] <= box[4])


def test_roi_atlas_attenuates_box_receivers_like_the_dense_atlas():
    occ, recv, lights, radii, box, H, W = _setup()
    dense = oracle.build_atlas(occ, lights, H, W, radii)
    mask, kr = oracle.f32_roi(recv.means, box, lights, H, W, radii)
    roi = oracle.roi_atlas(dense, mask, kr)
    inside = _in_box(recv.means, box)
    assert 200 < inside.sum() < recv.n  # a real subset
    c_d, T_d = oracle.attenuate(dense, radii, lights, recv.means[inside], recv.colors[inside], want_T=True)
    c_r, T_r = oracle.attenuate(roi, radii, lights, recv.means[inside], recv.colors[inside], want_T=True)
    assert np.array_equal(T_r, T_d) and np.array_equal(c_r, c_d)
    # the region is a small part of the atlas and it matters outside it
    assert mask.mean() < 0.6
    out = ~inside
    _, T_o = oracle.attenuate(roi, radii, lights, recv.means[out], recv.colors[out], want_T=True)
    _, T_od = oracle.attenuate(dense, radii, lights, recv.means[out], recv.colors[out], want_T=True)
    assert np.abs(T_o - T_od).max() > 1e-3


def test_roi_mask_is_the_set_of_lookup_taps():
    occ, recv, lights, radii, box, H, W = _setup(seed=3)
    mask, kr = oracle.f32_roi(recv.means, box, lights, H, W, radii)
    inside = recv.means[_in_box(recv.means, box)]
    K = radii.shape[0]
    for l in range(lights.shape[0]):
        oi, of = oracle.f32_sample_index(inside, lights[l], H, W, radii)
        keep = of[:, 2] != 0
        oi = oi[keep]
        ref = np.zeros((H, W), np.uint8)
        for di in (0, 1):
            for dj in (0, 1):
                ref[np.clip(oi[:, 2] + di, 0, H - 1), np.clip(oi[:, 3] + dj, 0, W - 1)] = 1
        assert np.array_equal(mask[l], ref)
        k = oi[:, 4]
        k0 = np.where(k < 0, 0, np.minimum(k, K - 1))
        k1 = np.where(k < 0, 0, np.minimum(k + 1, K - 1))
        assert (kr[l, 0], kr[l, 1]) == (k0.min(), k1.max())


def test_roi_box_closed_form():
    m = np.float32([[1.0, 2.0, 0.0], [3.0, -2.0, 1.5], [0.0, 0.0, 0.7]])
    a = np.float32([0.5, 0.25, 0.25])
    box = oracle.roi_box(m, a, R=2.0, z_margin=0.1)
    assert np.allclose(box, [0.5 * 1 + 0.25 * 3, 0.5 * 2 - 0.25 * 2, 2.0, -0.1, 1.6], rtol=0, atol=1e-12)


def test_roi_empty_cases():
    occ, recv, lights, radii, box, H, W = _setup(seed=5)
    K = radii.shape[0]
    empty = np.float32([0, 0, -1, 0, 0])  # R < 0: no receiver inside
    mask, kr = oracle.f32_roi(recv.means, empty, lights, H, W, radii)
    assert mask.sum() == 0 and (kr[:, 0] == K).all() and (kr[:, 1] == -1).all()
    dense = oracle.build_atlas(occ, lights, H, W, radii)
    assert (oracle.roi_atlas(dense, mask, kr) == 1).all()
    # a receiver at the light reads nothing
    mask, kr = oracle.f32_roi(lights[:1], np.float32([0, 0, 1, -1, 1]), lights[:1], H, W, radii)
    assert mask.sum() == 0 and kr[0, 1] == -1
