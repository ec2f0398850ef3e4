"""GPU parity of the local-PCA pseudo-normals (Sec. 4) against the FP64
oracle: surfaces (a tilted plane, a sphere), an avatar body and a mix with
isolated and coincident Gaussians (smallest-axis fallback), a sample of the
full room at its own size, and the argument checks.

Where the covariance's two smallest eigenvalues are well apart
((l1 - l0) >= 0.05 l2) the eigenvector is unique: the kernel's FP32 sums over
a few hundred neighbours perturb C by about 1e-6 l2, so the normal moves by
about 1e-6 / 0.05; the bound is 1e-4.  Elsewhere several directions are
(nearly) correct: the kernel's normal must be a unit vector whose weighted
second moment is within 1e-4 l2 of the smallest.  Fallback normals (the
smallest-scale axis) agree to 1e-5.  Where the normal lies in the plane
through the centroid (|n . (x - c)| < 1e-5) the sign is not compared."""
import numpy as np
import pytest
import torch

from oracle import normals as onorm
from paper_2601_01660_b300 import scenes

from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    return native()


def _compare(nat, x, op, quats, scales, r, c, idx=None):
    x, op = np.float32(x), np.float32(op)
    quats, scales = np.float32(quats), np.float32(scales)
    got = nat.dgsm_pca_normals(dev(x), dev(op), dev(quats), dev(scales), dev(np.float32(c)), radius=r)
    got = got.double().cpu().numpy()
    rows = np.arange(x.shape[0]) if idx is None else np.asarray(idx)
    got = got[rows]
    ref, lam, fb = onorm.pca_normals(x, op, quats, scales, float(np.float32(r)), c, want_info=True, idx=rows)
    assert np.abs(np.linalg.norm(got, axis=1) - 1).max() < 1e-5
    side = np.einsum("nc,nc->n", ref, x[rows].astype(np.float64) - np.asarray(c, np.float64))
    flip = np.where((np.abs(side) < 1e-5) & (np.einsum("nc,nc->n", got, ref) < 0), -1.0, 1.0)
    g = got * flip[:, None]
    assert np.abs(g[fb] - ref[fb]).max(initial=0) < 1e-5
    gap = (lam[:, 1] - lam[:, 0]) >= 0.05 * np.maximum(lam[:, 2], 1e-300)
    uniq = ~fb & gap
    assert np.abs(g[uniq] - ref[uniq]).max(initial=0) < 1e-4
    for k in np.nonzero(~fb & ~gap)[0]:
        _, _, C, _ = onorm.weighted_moments(x, op, rows[k], float(np.float32(r)))
        assert g[k] @ C @ g[k] <= lam[k, 0] + 1e-4 * lam[k, 2]
    return fb, uniq


def test_plane_sphere_and_avatar(nat):
    rng = np.random.default_rng(0)
    nu = np.array([0.3, -0.2, 1.0]) / np.linalg.norm([0.3, -0.2, 1.0])
    a = np.cross(nu, [1.0, 0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(nu, a)
    uv = rng.uniform(-0.5, 0.5, (1500, 2))
    plane = np.array([0.0, 0.0, 2.0]) + uv[:, :1] * a + uv[:, 1:] * b
    u = rng.normal(size=(1500, 3))
    sphere = np.array([2.0, 1.0, 1.0]) + 0.4 * u / np.linalg.norm(u, axis=1, keepdims=True)
    av = scenes.avatar_body(rng, 2000, base=(-1.0, 0.0, 0.0))
    x = np.concatenate([plane, sphere, av.means])
    n = x.shape[0]
    op = np.concatenate([rng.uniform(0.05, 1.0, 3000), av.opac])
    quats = np.concatenate([rng.normal(size=(3000, 4)), av.quats])
    scales = np.concatenate([np.exp(rng.normal(-3.5, 0.4, (3000, 3))), av.scales])
    c = np.array([0.3, 0.1, 1.2])
    fb, uniq = _compare(nat, x, op, quats, scales, 0.08, c)
    assert uniq[:1500].mean() > 0.95 and uniq.sum() > 0.7 * n


def test_isolated_and_coincident_fall_back(nat):
    rng = np.random.default_rng(1)
    far = rng.uniform(-20, 20, (300, 3))                   # isolated at r = 0.05
    dup = np.repeat(rng.uniform(-1, 1, (50, 3)), 4, axis=0)  # groups of four coincident centres
    cl = 0.3 * rng.normal(size=(400, 3)) * [1.0, 1.0, 0.05] + [5.0, 5.0, 5.0]   # a thin slab
    x = np.concatenate([far, dup, cl])
    n = x.shape[0]
    op = rng.uniform(0.1, 1.0, n)
    op[:10] = 0.0
    quats = rng.normal(size=(n, 4))
    scales = np.exp(rng.normal(-3, 0.5, (n, 3)))
    fb, _ = _compare(nat, x, op, quats, scales, 0.05, np.zeros(3))
    assert fb[:500].all()


def test_room_sample_at_full_size(nat):
    wl = scenes.workload("room1p6m")
    sc = wl["occluders"]
    sel = np.random.default_rng(2).choice(sc.n, 200, replace=False)
    sl = sc.meta["avatar"]
    sel = np.concatenate([sel, np.arange(sl.start, sl.stop, 1000)])  # and the avatar
    c = sc.means[sl].astype(np.float64).mean(0)
    fb, uniq = _compare(nat, sc.means, sc.opac, sc.quats, sc.scales, 0.05, c, idx=sel)
    assert uniq.mean() > 0.5


def test_empty_and_bad_arguments(nat):
    from paper_2601_01660_b300._native import DGSMError
    e = torch.empty((0, 3), device="cuda")
    out = nat.dgsm_pca_normals(e, torch.empty(0, device="cuda"), torch.empty((0, 4), device="cuda"), e,
                               dev([0, 0, 0]))
    assert out.shape == (0, 3)
    x = dev(np.float32([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0]]))
    q = dev(np.float32([[1, 0, 0, 0]] * 3))
    for r in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(DGSMError):
            nat.dgsm_pca_normals(x, dev([1, 1, 1]), q, x, dev([0, 0, 0]), radius=r)


def test_relight_with_pca_normals(nat, orc):
    """The pseudo-normals feed the relight (Eqs. 8-10): the avatar relit with
    its own PCA normals against the FP64 relight given the oracle's normals
    (the two normal sets agree to 1e-4 where unique, so the lobe sums agree
    to about 1e-3 relative)."""
    rng = np.random.default_rng(5)
    av = scenes.avatar_body(rng, 4000)
    c = av.means.astype(np.float64).mean(0)
    d = {k: dev(getattr(av, k)) for k in ("means", "opac", "quats", "scales", "colors")}
    nrm = nat.dgsm_pca_normals(d["means"], d["opac"], d["quats"], d["scales"], dev(np.float32(c)), radius=0.08)
    D, Y, w = scenes.cubemap_samples(32, seed=5)
    sh = orc.sh_fit(D, Y, w)
    out = nat.sh_relight(dev(sh), d["means"], d["quats"], d["scales"], d["colors"], dev(np.float32(c)),
                         normals=nrm).double().cpu().numpy()
    ref_n, lam, fb = onorm.pca_normals(av.means, av.opac, av.quats, av.scales, float(np.float32(0.08)), c,
                                      want_info=True)
    ref = orc.relight(sh, av, c, normals=np.float32(ref_n))
    uniq = fb | ((lam[:, 1] - lam[:, 0]) >= 0.05 * lam[:, 2])
    err = np.abs(out - ref) / np.maximum(np.abs(ref), 1e-6)
    assert uniq.mean() > 0.7 and err[uniq].max() <= 2e-3
