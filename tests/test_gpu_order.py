"""GPU tests of the scene storage order (dgsm_spatial_order,
dgsm_gather_rows): the permutation sorts the Z-order codes as the header
defines them (recomputed here in float32 numpy, bit for bit), stably; rows
gather exactly; and the method's results do not depend on the order (the
attenuation of a receiver bit for bit, the atlas up to the order of its
sums)."""
import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import layout, scenes

from gpu_util import dev, scene_to_dev

pytestmark = pytest.mark.gpu

DGSM_ERR_INVALID_ARG = 1


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _spread(q):
    code = np.zeros(q.shape[0], np.uint64)
    for b in range(10):
        code |= ((q >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return code


def zorder_codes(means):
    """The codes of the header's definition: cells of a 1024^3 grid over the
    bounding box, each float operation rounded once (numpy float32 is IEEE
    single precision, rounded to nearest)."""
    m = np.asarray(means, np.float32)
    lo, hi = m.min(0), m.max(0)
    code = np.zeros(m.shape[0], np.uint64)
    with np.errstate(invalid="ignore", divide="ignore"):
        for a in range(3):
            ext = np.float32(hi[a] - lo[a])
            inv = np.float32(np.float32(1024.0) / ext) if ext > 0 else np.float32(0.0)
            f = np.floor(np.float32(m[:, a] - lo[a]) * inv)
            q = np.clip(np.nan_to_num(f, nan=0.0), 0, 1023).astype(np.uint64)
            code |= _spread(q) << np.uint64(a)
    return code


def _check_perm(perm, n):
    assert perm.dtype == np.int32 and perm.shape == (n,)
    assert np.array_equal(np.sort(perm), np.arange(n))


@pytest.mark.parametrize("n", [1, 2, 1000, 300_001])
def test_order_sorts_the_codes_stably(nat, n):
    rng = np.random.default_rng(n)
    m = rng.normal(size=(n, 3)).astype(np.float32) * np.float32([4.0, 3.0, 1.0])
    if n > 10:
        m[::7] = m[3]  # repeated means: equal codes keep their index order
    perm = nat.dgsm_spatial_order(dev(m)).cpu().numpy()
    _check_perm(perm, n)
    want = np.argsort(zorder_codes(m), kind="stable")
    assert np.array_equal(perm, want)


def test_order_flat_axis_and_non_finite_means(nat):
    rng = np.random.default_rng(3)
    m = rng.random((5000, 3)).astype(np.float32)
    m[:, 2] = 0.25  # a flat axis
    perm = nat.dgsm_spatial_order(dev(m)).cpu().numpy()
    assert np.array_equal(perm, np.argsort(zorder_codes(m), kind="stable"))
    m[17, 0] = np.nan
    m[99, 1] = np.inf
    perm = nat.dgsm_spatial_order(dev(m)).cpu().numpy()
    _check_perm(perm, m.shape[0])
    assert nat.dgsm_sync_status() == 0
    empty = nat.dgsm_spatial_order(torch.empty((0, 3), device="cuda"))
    assert empty.shape == (0,)


def test_gather_rows(nat):
    rng = np.random.default_rng(5)
    src = dev(rng.random((1234, 3)))
    perm = torch.as_tensor(rng.permutation(1234)[:1000].astype(np.int32)).cuda()
    out = nat.dgsm_gather_rows(src, perm)
    assert torch.equal(out, src[perm.long()])
    q = dev(rng.random((50, 4)))
    p2 = torch.arange(49, -1, -1, dtype=torch.int32, device="cuda")
    assert torch.equal(nat.dgsm_gather_rows(q, p2), q.flip(0))
    o1 = dev(rng.random(77))
    p3 = torch.arange(77, dtype=torch.int32, device="cuda")
    assert torch.equal(nat.dgsm_gather_rows(o1, p3), o1)
    # an entry out of range: its row is zero and the status reports it
    bad = perm.clone()
    bad[10] = 1234
    torch.cuda.synchronize()
    out = nat.dgsm_gather_rows(src, bad)
    torch.cuda.synchronize()
    assert nat.dgsm_sync_status() == DGSM_ERR_INVALID_ARG
    assert bool((out[10] == 0).all())
    assert torch.equal(out[:10], src[perm[:10].long()])


def test_results_do_not_depend_on_the_order(nat):
    """The same scene in scene order and in Z-order: the atlas agrees to the
    order of its sums, and each receiver's attenuated colour bit for bit."""
    sc = scenes.cube_scene(20000, seed=11, log_s_mean=np.log(0.03))
    zc, perm = layout.zorder_scene(nat, sc, [0, 5000, sc.n], "cuda")
    assert np.array_equal(np.sort(perm[:5000]), np.arange(5000))
    lights = dev(np.float32([[0.0, 0.0, 0.0], [0.4, -0.3, 0.2]]))
    radii = dev(scenes.radii_geometric(0.05, 4.0, 32))
    a = scene_to_dev(sc)
    b = scene_to_dev(zc)
    A = nat.dgsm_build(a["means"], a["scales"], a["quats"], a["opac"], lights, 128, 128, radii)
    B = nat.dgsm_build(b["means"], b["scales"], b["quats"], b["opac"], lights, 128, 128, radii)
    assert float(A.min()) < 0.5
    assert torch.allclose(A, B, atol=2e-6, rtol=0)
    ca = nat.dgsm_attenuate(A, radii, lights, a["means"], a["colors"])
    cb = nat.dgsm_attenuate(A, radii, lights, b["means"], b["colors"])
    assert torch.equal(cb, ca[torch.as_tensor(perm).cuda()])
    assert nat.dgsm_sync_status() == 0
