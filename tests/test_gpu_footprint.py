"""GPU parity of footprint attenuation (Sec. 3.3 last paragraph; ablation (A)
of Sec. 4): the 7-point stencil and the Monte Carlo footprint (Philox4x64-10
offsets generated in the kernel) against the FP64 oracle on the same atlas,
at small sizes over several blocks with a ragged tail and at the benchmark's
full size on sampled receivers.

Tolerance: the kernel forms each sample point and its octahedral index in
FP32 (the oracle in FP64), about 2e-7 m of rounding at 3 m from the light;
the Monte Carlo offsets differ by a few FP32 ulps of Box-Muller.  The
trilinear lookup is continuous, so T moves by that distance times its
gradient, at most ~0.5 per texel (~6 mm at 3 m on a 512 atlas): a few 1e-5,
inside |dT| <= 1e-4."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


@pytest.fixture(scope="module")
def small(nat):
    sc = scenes.cube_scene(1500, seed=0)
    lights = np.float32([[0, 0, 0], [0.5, -0.5, 1.0]])
    radii = scenes.radii_linear(0.1, 8, 8)
    H, W = 24, 40
    d = scene_to_dev(sc)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii))
    q = scenes.cube_scene(5000, seed=1)  # 5000 = 39 blocks of 128 + a ragged tail
    return sc, lights, radii, atlas, q


@pytest.mark.parametrize("mode,n", [("stencil7", 7), ("mc", 8), ("mc", 1), ("mc", 32)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_footprint_matches_oracle(nat, orc, small, mode, n, dtype):
    sc, lights, radii, atlas, q = small
    at = atlas.to(dtype)
    lw = np.float32([0.3, 0.7])
    out, T = nat.dgsm_attenuate_footprint(at, dev(radii), dev(lights), dev(q.means), dev(q.quats),
                                          dev(q.scales), dev(q.colors), mode=mode, n_samples=n, seed=7,
                                          light_w=dev(lw), direct_frac=0.8, want_T=True)
    ref, Tref = orc.attenuate_footprint(at.double().cpu().numpy(), radii, lights, q.means, q.quats,
                                        q.scales, q.colors, mode=mode, n_samples=n, seed=7,
                                        light_w=lw, direct_frac=0.8, want_T=True)
    err = np.abs(T.double().cpu().numpy() - Tref)
    assert err.max() <= TOL and np.median(err) <= 1e-6, err.max()
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL
    assert Tref.min() < 0.9  # the receivers see real shadow


def test_footprint_centre_equals_centre_lookup(nat, small):
    """The footprint pass's centre mode is the centre lookup; the streamed
    centre-lookup kernel rounds its interpolation in another order (lerps,
    and d2 rsqrt(d2) for t in the shell weight), so the two agree to a few
    ulps rather than bit for bit."""
    sc, lights, radii, atlas, q = small
    args = (atlas, dev(radii), dev(lights), dev(q.means))
    c0, T0 = nat.dgsm_attenuate(*args, dev(q.colors), want_T=True)
    c1, T1 = nat.dgsm_attenuate_footprint(*args, dev(q.quats), dev(q.scales), dev(q.colors),
                                          mode="centre", want_T=True)
    assert torch.allclose(T0, T1, atol=1e-6, rtol=0) and torch.allclose(c0, c1, atol=1e-6, rtol=0)


def test_footprint_seed_and_in_place(nat, small):
    sc, lights, radii, atlas, q = small
    args = (atlas, dev(radii), dev(lights), dev(q.means), dev(q.quats), dev(q.scales))
    _, Ta = nat.dgsm_attenuate_footprint(*args, dev(q.colors), seed=1, want_T=True)
    _, Tb = nat.dgsm_attenuate_footprint(*args, dev(q.colors), seed=1, want_T=True)
    _, Tc = nat.dgsm_attenuate_footprint(*args, dev(q.colors), seed=2, want_T=True)
    assert torch.equal(Ta, Tb)           # counter-based: the same seed repeats exactly
    assert not torch.equal(Ta, Tc)
    col = dev(q.colors)
    ref = nat.dgsm_attenuate_footprint(*args, col.clone(), seed=1)
    nat.dgsm_attenuate_footprint(*args, col, seed=1, out=col)  # colours_out == colours_in
    assert torch.equal(col, ref)


def test_footprint_edge_cases(nat, small):
    sc, lights, radii, atlas, q = small
    e = lambda a: dev(np.zeros((0, a), np.float32))
    out = nat.dgsm_attenuate_footprint(atlas, dev(radii), dev(lights), e(3), e(4), e(3), e(3))
    assert out.shape == (0, 3)
    # receivers at a light and beyond the last shell
    qm = np.float32([[0, 0, 0], [0.5, -0.5, 1.0], [40, 0, 0]])
    qq = np.float32([[1, 0, 0, 0]] * 3)
    qs = np.float32([[1e-3] * 3] * 3)
    _, T = nat.dgsm_attenuate_footprint(atlas, dev(radii), dev(lights), dev(qm), dev(qq), dev(qs),
                                        dev(np.ones((3, 3), np.float32)), mode="stencil7", want_T=True)
    assert torch.isfinite(T).all() and (T >= 0).all() and (T <= 1.0 + 1e-6).all()
    from paper_2601_01660_b300._native import DGSMError
    for kw in ({"mode": "mc", "n_samples": 0}, {"mode": "mc", "n_samples": 33}):
        with pytest.raises(DGSMError):
            nat.dgsm_attenuate_footprint(atlas, dev(radii), dev(lights), dev(q.means), dev(q.quats),
                                         dev(q.scales), dev(q.colors), **kw)


def test_room_footprint_sampled_receivers(nat, orc):
    """The benchmark's room workload: MC footprint (8 samples) of all 1.6M
    Gaussians, checked on 2000 sampled receivers."""
    wl = scenes.workload("room1p6m")
    sc = wl["occluders"]
    d = scene_to_dev(sc)
    lights, radii = dev(wl["lights"]), dev(wl["radii"])
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lights, wl["H"], wl["W"], radii)
    out, T = nat.dgsm_attenuate_footprint(atlas, radii, lights, d["means"], d["quats"], d["scales"],
                                          d["colors"], mode="mc", n_samples=8, seed=3, want_T=True)
    idx = np.sort(np.random.default_rng(21).choice(sc.n, 2000, replace=False))
    ref, Tref = orc.attenuate_footprint(atlas.double().cpu().numpy(), wl["radii"], wl["lights"],
                                        sc.means[idx], sc.quats[idx], sc.scales[idx], sc.colors[idx],
                                        mode="mc", n_samples=8, seed=3, want_T=True, q_ids=idx)
    err = np.abs(T.double().cpu().numpy()[idx] - Tref)
    assert err.max() <= TOL and np.median(err) <= 1e-6, err.max()
    assert np.abs(out.double().cpu().numpy()[idx] - ref).max() <= TOL
