"""GPU parity of the DGSM build (Sec. 3.2) and its binning through the C ABI,
against the FP64 oracle and the oracle's FP32 binning specification."""
import math

import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

from gpu_util import dev, scene_to_dev, texel_sample

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-4             # |dT| for float32 storage
TOL_F16 = 2e-3             # |dT| for float16 storage (half ulp 2^-12 near 1, plus build error)
TOL_BF16 = 2.0 ** -9 + 1e-4  # bfloat16 storage: half ulp of T in [0.5, 1) plus build error


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _build(nat, sc, lights, H, W, radii, **params):
    d = scene_to_dev(sc)
    return nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W,
                          dev(radii), params=params)


@pytest.mark.parametrize("H,W,tile,nl", [(32, 32, 8, 1), (44, 60, 8, 2), (64, 48, 16, 1),
                                         (40, 40, 4, 3), (128, 128, 8, 1)])
def test_binning_bit_exact(nat, orc, H, W, tile, nl):
    rng = np.random.default_rng(H)
    cube = scenes.cube_scene(2500, seed=31 + H, log_s_mean=math.log(0.06))
    flat = scenes.cube_scene(1500, seed=32 + H, log_s_mean=math.log(0.1))
    flat.scales[np.arange(flat.n), rng.integers(0, 3, flat.n)] = 0.002   # 2 mm thick discs
    sc = scenes.concat(cube, flat, scenes.avatar_body(rng, 1000, base=(0.3, 0.2, 1.5)))
    lights = np.float32([[0, 0, 0], [0.4, -0.3, 0.5], [-1, 1, 2.5]])[:nl]
    radii = scenes.radii_linear(0.1, 8, 10)
    ko, vo = orc.f32_bin(sc, lights, H, W, radii, eps=1e-7, tile=tile)
    d = scene_to_dev(sc)
    kg, vg = nat.dgsm_bin(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii),
                          params=dict(tile=tile))
    assert kg.numel() == ko.size
    assert np.array_equal(kg.cpu().numpy().astype(np.uint32), ko)
    assert np.array_equal(vg.cpu().numpy().astype(np.uint32), vo)


def test_binning_light_inside_and_beyond_shells(nat, orc):
    """Gaussians around the light (bound to every tile) and beyond the last
    shell (bound nowhere) follow the specification too."""
    sc = scenes.cube_scene(1500, seed=41, centre=(0, 0, 0), side=12.0, log_s_mean=math.log(0.2))
    lights = np.float32([[0.05, 0.0, -0.02]])
    radii = scenes.radii_linear(0.1, 3.0, 6)
    ko, vo = orc.f32_bin(sc, lights, 24, 24, radii)
    d = scene_to_dev(sc)
    kg, vg = nat.dgsm_bin(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), 24, 24, dev(radii))
    assert np.array_equal(kg.cpu().numpy().astype(np.uint32), ko)
    assert np.array_equal(vg.cpu().numpy().astype(np.uint32), vo)


@pytest.mark.parametrize("H,W,tile,K,chunk", [(44, 60, 8, 12, 64), (32, 32, 16, 7, 16),
                                               (20, 36, 8, 5, 16), (40, 24, 8, 9, 32), (48, 40, 8, 10, 192),
                                               (32, 48, 16, 6, 160)])
def test_build_matches_oracle_every_voxel(nat, orc, H, W, tile, K, chunk):
    """Small chunks cut long tile lists into several work items, so this also
    covers the cross-item accumulation."""
    sc = scenes.cube_scene(3000, seed=5 + K)
    lights = np.float32([[0, 0, 0], [0.3, -0.2, 0.4]])
    radii = scenes.radii_linear(0.1, 8, K)
    T_ref = orc.build_atlas(sc, lights, H, W, radii)
    T = _build(nat, sc, lights, H, W, radii, tile=tile, chunk=chunk).double().cpu().numpy()
    err = np.abs(T - T_ref)
    assert err.max() <= TOL_F32, (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("radii", [[3.0], [1.5, 4.0], [0.4, 2.5, 6.0], [2.0, 2.05, 2.1, 5.5]])
def test_build_few_shells_matches_oracle(nat, orc, radii):
    """One to three shells (the shell table and the shell loop read the radii
    up to two places past the last, which hold +inf), and radii closer than
    the table's buckets (the shells then counted one by one)."""
    sc = scenes.cube_scene(2500, seed=31 + len(radii))
    lights = np.float32([[0, 0, 0], [0.2, 0.3, -0.1]])
    radii = np.float32(radii)
    T_ref = orc.build_atlas(sc, lights, 24, 40, radii)
    T = _build(nat, sc, lights, 24, 40, radii, chunk=32).double().cpu().numpy()
    err = np.abs(T - T_ref)
    assert err.max() <= TOL_F32, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert (T < 0.999).any()  # the shells hold shadow


@pytest.mark.parametrize("dtype,tol", [("f16", TOL_F16), ("bf16", TOL_BF16)])
def test_build_half_storage(nat, orc, dtype, tol):
    sc = scenes.cube_scene(2000, seed=77)
    lights = np.float32([[0, 0, 0]])
    radii = scenes.radii_geometric(0.05, 12, 9)
    T_ref = orc.build_atlas(sc, lights, 40, 40, radii)
    T = _build(nat, sc, lights, 40, 40, radii, atlas_dtype=dtype)
    assert T.dtype == {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    assert np.abs(T.double().cpu().numpy() - T_ref).max() <= tol


def test_build_empty_and_transparent(nat):
    radii = scenes.radii_linear(0.1, 8, 5)
    sc = scenes.cube_scene(0, seed=0)
    T = _build(nat, sc, np.float32([[0, 0, 0]]), 16, 24, radii)
    assert T.shape == (1, 5, 16, 24) and bool((T == 1).all())
    sc = scenes.cube_scene(500, seed=1)
    sc.opac[:] = 0
    T = _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, radii)
    assert bool((T == 1).all())


def test_build_bounds_and_monotone(nat):
    sc = scenes.cube_scene(20_000, seed=0)
    T = _build(nat, sc, np.float32([[0, 0, 0]]), 64, 64, scenes.radii_linear(0.1, 8, 16))
    assert bool(((T >= 0) & (T <= 1)).all())
    assert bool((T[:, 1:] <= T[:, :-1]).all())


def test_build_cube20k_sampled(nat, orc):
    """The 20k-Gaussian cube workload at full size (64x64x16, one light at
    the origin), checked on 256 random texels x all shells."""
    wl = scenes.workload("cube20k")
    sc, lights, radii = wl["occluders"], wl["lights"], wl["radii"]
    T = _build(nat, sc, lights, 64, 64, radii).double().cpu().numpy()
    lij = texel_sample(np.random.default_rng(0), 1, 64, 64, 256)
    tau = orc.build_tau_texels(sc, lights, 64, 64, radii, lij)
    got = T[lij[:, 0], :, lij[:, 1], lij[:, 2]]
    assert np.abs(got - np.exp(-tau)).max() <= TOL_F32


def test_build_stats_are_consistent(nat):
    sc = scenes.cube_scene(5000, seed=3)
    _build(nat, sc, np.float32([[0, 0, 0]]), 64, 64, scenes.radii_linear(0.1, 8, 16))
    st = nat.dgsm_get_build_stats()
    assert st["n_pairs"] > 0
    assert 0 < st["ray_evals"] <= st["rays_tested"] <= 64 * st["n_pairs"]


@pytest.mark.parametrize("workload", ["cube", "room_shapes"])
def test_ray_evals_match_oracle_count(nat, orc, workload):
    """The throughput metric's unit, the Gaussian-ray evaluations (pairs whose
    ray cuts the Gaussian's culling ellipsoid ahead of the light), counted by
    the GPU build equals the oracle's FP64 count over every texel, up to the
    pairs that sit on the ellipsoid's boundary (float32 against float64
    decides them; a few in 10^4)."""
    if workload == "cube":
        sc = scenes.cube_scene(4000, seed=21)
        lights = np.float32([[0, 0, 0], [0.4, -0.3, 0.6]])
    else:
        rng = np.random.default_rng(22)
        sc = scenes.cube_scene(3000, seed=23, log_s_mean=math.log(0.08))
        sc.scales[np.arange(sc.n), rng.integers(0, 3, sc.n)] = 0.002  # 2 mm thick discs
        lights = np.float32([[0.1, -0.2, 0.3]])
    H, W = 40, 56
    radii = scenes.radii_geometric(0.05, 12, 12)
    _build(nat, sc, lights, H, W, radii)
    got = nat.dgsm_get_build_stats()["ray_evals"]
    L = lights.shape[0]
    lij = np.stack(np.meshgrid(np.arange(L), np.arange(H), np.arange(W), indexing="ij"), -1).reshape(-1, 3)
    ref = orc.count_ray_evals(sc, lights, H, W, radii, lij)
    assert ref > 10_000
    assert abs(got - ref) <= 5e-4 * ref + 2, (got, ref)


def test_nonfinite_input_is_reported(nat):
    sc = scenes.cube_scene(100, seed=2)
    sc.means[7, 1] = np.nan
    with pytest.raises(nat.DGSMError) as ei:
        _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4))
    assert ei.value.code == 5
    sc = scenes.cube_scene(100, seed=2)
    sc.scales[3, 0] = 0.0
    with pytest.raises(nat.DGSMError):
        _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4))
    # the context stays usable
    sc = scenes.cube_scene(100, seed=2)
    T = _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4))
    assert bool(torch.isfinite(T).all())


def test_bad_arguments_are_rejected(nat):
    sc = scenes.cube_scene(10, seed=2)
    with pytest.raises(nat.DGSMError) as ei:
        _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4), tile=5)
    assert ei.value.code == 1
    with pytest.raises(nat.DGSMError):
        _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4), chunk=4)
    with pytest.raises(nat.DGSMError):   # three staging loads per thread hold at most 192 records
        _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4), chunk=193)
    with pytest.raises(nat.DGSMError):   # 4x4 tiles: binning only
        _build(nat, sc, np.float32([[0, 0, 0]]), 16, 16, scenes.radii_linear(0.1, 8, 4), tile=4)


def test_maximum_sizes(nat, orc):
    """The largest sizes the build accepts: 256 shells; a 4096 x 4096 atlas
    (sampled texels); 64 lights.  Each against the FP64 oracle."""
    sc = scenes.cube_scene(600, seed=21)
    # K = 256 geometric shells on a small atlas, every voxel
    radii = scenes.radii_geometric(0.05, 12.0, 256)
    T = _build(nat, sc, np.float32([[0, 0, 0]]), 12, 12, radii).double().cpu().numpy()
    assert np.abs(T - orc.build_atlas(sc, np.float32([[0, 0, 0]]), 12, 12, radii)).max() <= TOL_F32
    # H = W = 4096 (2 shells), 300 random texels
    radii2 = np.float32([0.5, 9.0])
    T = _build(nat, sc, np.float32([[0.1, 0.2, 0.3]]), 4096, 4096, radii2)
    lij = texel_sample(np.random.default_rng(1), 1, 4096, 4096, 300)
    got = T[lij[:, 0], :, lij[:, 1], lij[:, 2]].double().cpu().numpy()
    tau = orc.build_tau_texels(sc, np.float32([[0.1, 0.2, 0.3]]), 4096, 4096, radii2, lij)
    assert np.abs(got - np.exp(-tau)).max() <= TOL_F32 and np.exp(-tau).min() < 0.99
    # 64 lights, every voxel
    lights = np.float32(np.random.default_rng(2).uniform(-2, 2, (64, 3)) + [0, 0, 3.0])
    radii3 = scenes.radii_linear(0.1, 8, 4)
    T = _build(nat, sc, lights, 8, 8, radii3).double().cpu().numpy()
    assert np.abs(T - orc.build_atlas(sc, lights, 8, 8, radii3)).max() <= TOL_F32
    with pytest.raises(nat.DGSMError):   # one past each limit
        _build(nat, sc, np.float32([[0, 0, 0]]), 8, 8, scenes.radii_geometric(0.05, 12.0, 257))
    with pytest.raises(nat.DGSMError):
        _build(nat, sc, np.float32([[0, 0, 0]]), 4097, 8, radii2)
    with pytest.raises(nat.DGSMError):
        _build(nat, sc, np.zeros((65, 3), np.float32), 8, 8, radii2)


@pytest.mark.parametrize("tile,nl,amap", [(8, 3, 0), (16, 2, 0), (8, 2, 1)])
def test_build_bins_the_same_pairs_as_dgsm_bin(nat, tile, nl, amap):
    """dgsm_build writes its super-tile lists unsorted (from per-(light,
    Gaussian) super-tile masks and per-block ranges) while dgsm_bin sorts
    them; both take the same decisions, so the pair counts at both levels are
    equal (dgsm_bin's pairs are the bit-exact specification)."""
    rng = np.random.default_rng(5 + tile + nl)
    cube = scenes.cube_scene(3000, seed=51, log_s_mean=math.log(0.06))
    flat = scenes.cube_scene(2000, seed=52, log_s_mean=math.log(0.1))
    flat.scales[np.arange(flat.n), rng.integers(0, 3, flat.n)] = 0.002
    sc = scenes.concat(cube, flat, scenes.avatar_body(rng, 1500, base=(0.3, 0.2, 1.5)))
    lights = np.float32([[0, 0, 0], [0.4, -0.3, 0.5], [-1, 1, 2.5]])[:nl]
    radii = scenes.radii_linear(0.1, 8, 10)
    H, W = (96, 128) if amap == 0 else (6 * 32, 32)
    params = dict(tile=tile, atlas_map=amap)
    d = scene_to_dev(sc)
    keys, _ = nat.dgsm_bin(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii),
                           params=params)
    st_bin = nat.dgsm_get_build_stats()
    nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], dev(lights), H, W, dev(radii), params=params)
    st_build = nat.dgsm_get_build_stats()
    assert nat.dgsm_sync_status() == 0
    assert st_build["n_pairs"] == keys.numel() > 1000
    assert st_build["n_super_pairs"] == st_bin["n_super_pairs"] > 0
