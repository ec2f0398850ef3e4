"""FP64 CPU oracle for the Deep Gaussian Shadow Map hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only code that may import this package.
The product path (paper_2601_01660_b300) never imports it, and it never
imports the product path: both take their inputs from the seeded generators
in paper_2601_01660_b300.scenes, which hold none of the method's arithmetic.

The arithmetic lives in dgsm_oracle.c (plain C, FP64, OpenMP), one function
per equation of the paper; this module only marshals numpy arrays.

Pinned by tests/test_oracle_*.py (quadrature of Eq. 2, the isotropic closed
form of Eqs. 3+5, empty scene, bounds and monotonicity of T, octahedral round
trip, SH orthonormality against scipy, exact recovery of band-limited
signals, the clamped-cosine irradiance limit of Eq. 10).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_SANITIZED=1 loads the ASan/UBSan build (its runtime must be preloaded)
        path = _build.build(sanitize=os.environ.get("ORACLE_SANITIZED") == "1")
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


_f = C.POINTER(C.c_float)
_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_u32 = C.POINTER(C.c_uint32)
I64 = C.c_int64


def _declare(L):
    L.orc_num_threads.restype = C.c_int
    L.orc_beta.restype = C.c_double
    L.orc_beta.argtypes = [_f, C.c_float, C.c_double]
    L.orc_line_integral.restype = C.c_double
    L.orc_line_integral.argtypes = [C.c_double] * 4
    L.orc_precision.argtypes = [_f, _f, _d]
    L.orc_quat_to_rot.argtypes = [_f, _d]
    L.orc_ray_coeffs.argtypes = [_d, _d, _d, _d, _d, _d]
    L.orc_octa_encode.argtypes = [_d, _d, _d]
    L.orc_octa_decode.argtypes = [C.c_double, C.c_double, _d]
    L.orc_texel_dir.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _d]
    L.orc_cube_encode.restype = C.c_int
    L.orc_cube_encode.argtypes = [_d, _d, _d]
    L.orc_cube_decode.argtypes = [C.c_int, C.c_double, C.c_double, _d]
    L.orc_build_tau.argtypes = [_f, _f, _f, _f, I64, _f, C.c_int, C.c_int, C.c_int, _f,
                                C.c_int, C.c_double, _d]
    L.orc_build_tau_texels.argtypes = [_f, _f, _f, _f, I64, _f, C.c_int, C.c_int, _f, C.c_int,
                                       C.c_double, _i32, I64, _d]
    L.orc_tau_rays.argtypes = [_f, _f, _f, _f, I64, _d, _d, _d, I64, C.c_double, _d]
    L.orc_sample_T.restype = C.c_double
    L.orc_sample_T.argtypes = [_d, C.c_int, C.c_int, _f, C.c_int, _d, _d]
    L.orc_attenuate.argtypes = [_d, _d, C.c_int, C.c_int, C.c_int, _f, C.c_int, _f, _f, _f, I64,
                                _f, C.c_double, _d, _d]
    L.orc_f32_sample_index_batch.argtypes = [_f, I64, _f, C.c_int, C.c_int, _f, C.c_int, _i32, _f]
    L.orc_f32_rect_cone.argtypes = [C.c_int] * 6 + [_f]
    L.orc_f32_gauss_cone.restype = C.c_int
    L.orc_f32_gauss_cone.argtypes = [_f, _f, C.c_float, _f, C.c_float, C.c_float, C.c_float, _f]
    L.orc_f32_bin.restype = I64
    L.orc_f32_rect_planes.argtypes = [C.c_int] * 7 + [_f]
    L.orc_f32_gauss_axes.argtypes = [_f, _f, _f, _f, _f]
    L.orc_f32_bin.argtypes = [_f, _f, _f, _f, I64, _f, C.c_int, C.c_int, C.c_int, _f, C.c_int,
                              C.c_float, C.c_float, C.c_int, _u32, _u32, I64]
    L.orc_f32_bin_keys.restype = I64
    L.orc_f32_bin_keys.argtypes = [_f, _f, _f, _f, I64, _f, C.c_int, C.c_int, C.c_int, _f, C.c_int,
                                   C.c_float, C.c_float, C.c_int, _u32, C.c_int, _u32, _u32, I64]
    L.orc_count_ray_evals.restype = I64
    L.orc_count_ray_evals.argtypes = [_f, _f, _f, _f, I64, _f, C.c_int, C.c_int, _f, C.c_int,
                                      C.c_float, C.c_float, _i32, I64]
    _u64 = C.POINTER(C.c_uint64)
    L.orc_philox4x64.argtypes = [_u64, _u64, _u64]
    L.orc_fp_normal.restype = C.c_double
    L.orc_fp_normal.argtypes = [C.c_uint64, I64, C.c_int]
    L.orc_fp_offsets.restype = C.c_int
    L.orc_fp_offsets.argtypes = [C.c_int, C.c_int, C.c_uint64, I64, _d, _d]
    L.orc_attenuate_footprint.argtypes = [_d, C.c_int, C.c_int, C.c_int, _f, C.c_int, _f, _f, _f, _f,
                                          _f, I64, _f, C.c_double, C.c_int, C.c_int, C.c_uint64,
                                          C.POINTER(C.c_int64), _d, _d]
    L.orc_f32_roi.argtypes = [_f, I64, _f, _f, C.c_int, C.c_int, C.c_int, _f, C.c_int,
                              C.POINTER(C.c_uint8), _i32]
    L.orc_set_beta_mode.argtypes = [C.c_int]
    L.orc_get_beta_mode.restype = C.c_int
    L.orc_set_atlas_map.argtypes = [C.c_int]
    L.orc_get_atlas_map.restype = C.c_int
    L.orc_render_pixels.argtypes = [_f, _f, _f, _f, _f, I64, _f, C.c_int, C.c_float,
                                    C.POINTER(C.c_int64), I64, _d]
    L.orc_render_view_pixels.argtypes = [_f, _f, _f, _f, _f, I64, _f, C.c_int, C.c_int, C.c_int, C.c_float,
                                         C.POINTER(C.c_int64), I64, _d]
    L.orc_cube_cams.argtypes = [_f, C.c_int, _f]
    L.orc_sh_basis.argtypes = [_d, _d]
    L.orc_sh_fit.restype = C.c_int
    L.orc_sh_fit.argtypes = [_f, _f, _f, I64, C.c_double, _d]
    L.orc_gauss_normal.argtypes = [_f, _f, _f, _f, _d]
    L.orc_transfer_scale.argtypes = [_d, _d, C.c_double, C.c_double, C.c_double, C.c_int,
                                     C.c_int, _d]
    L.orc_relight.argtypes = [_d, _f, _f, _f, _f, _f, _f, I64, C.c_double, C.c_double,
                              C.c_double, C.c_double, C.c_int, C.c_int, _d]


def _pf(a):
    return a.ctypes.data_as(_f) if a is not None else None


def _pd(a):
    return a.ctypes.data_as(_d) if a is not None else None


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# --- Gaussian parameters (Sec. 3.2, Eq. 5) --------------------------------

def precision(scale, quat) -> np.ndarray:
    A = np.zeros(9)
    lib().orc_precision(_pf(_c32(scale)), _pf(_c32(quat)), _pd(A))
    return A.reshape(3, 3)


def rotation(quat) -> np.ndarray:
    R = np.zeros(9)
    lib().orc_quat_to_rot(_pf(_c32(quat)), _pd(R))
    return R.reshape(3, 3)


class beta_mode:
    """Context manager: the oracle's opacity-to-absorption mapping (1..4; 2 is Eq. 5)."""

    def __init__(self, mode: int):
        if mode not in (1, 2, 3, 4):
            raise ValueError("beta mode must be 1..4")
        self.mode = mode

    def __enter__(self):
        self.prev = lib().orc_get_beta_mode()
        lib().orc_set_beta_mode(self.mode)
        return self

    def __exit__(self, *exc):
        lib().orc_set_beta_mode(self.prev)
        return False


class atlas_map:
    """Context manager: the oracle's atlas parameterisation, 0 the octahedral
    map (Sec. 3.2) or 1 the cube map (six F x F faces stacked in rows, H = 6F,
    W = F; the ablation's alternative)."""

    def __init__(self, map_id: int):
        if map_id not in (0, 1):
            raise ValueError("atlas map must be 0 (octahedral) or 1 (cube)")
        self.map_id = map_id

    def __enter__(self):
        self.prev = lib().orc_get_atlas_map()
        lib().orc_set_atlas_map(self.map_id)
        return self

    def __exit__(self, *exc):
        lib().orc_set_atlas_map(self.prev)
        return False


def beta(scale, alpha: float, kappa: float = 1.0) -> float:
    return float(lib().orc_beta(_pf(_c32(scale)), float(alpha), float(kappa)))


def ray_coeffs(A, d, o_minus_mu):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_ray_coeffs(_pd(_c64(A)), _pd(_c64(d)), _pd(_c64(o_minus_mu)),
                         C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def line_integral(a, b, c, t) -> float:
    """Eq. 3 (three-case erfc form)."""
    return float(lib().orc_line_integral(float(a), float(b), float(c), float(t)))


# --- octahedral map (Eq. 6) -------------------------------------------------

def octa_encode(d):
    u, v = C.c_double(), C.c_double()
    lib().orc_octa_encode(_pd(_c64(d)), C.byref(u), C.byref(v))
    return u.value, v.value


def octa_decode(u, v) -> np.ndarray:
    d = np.zeros(3)
    lib().orc_octa_decode(float(u), float(v), _pd(d))
    return d


def cube_encode(d):
    """(face, u, v) of direction d on the cube map."""
    u, v = C.c_double(), C.c_double()
    f = lib().orc_cube_encode(_pd(_c64(d)), C.byref(u), C.byref(v))
    return f, u.value, v.value


def cube_decode(f, u, v) -> np.ndarray:
    d = np.zeros(3)
    lib().orc_cube_decode(int(f), float(u), float(v), _pd(d))
    return d


def texel_dir(i, j, H, W) -> np.ndarray:
    d = np.zeros(3)
    lib().orc_texel_dir(int(i), int(j), int(H), int(W), _pd(d))
    return d


# --- DGSM build (Eqs. 1-5), brute force -------------------------------------

def build_tau(sc, lights, H, W, radii, kappa=1.0) -> np.ndarray:
    """tau[L][K][H][W] summed over every Gaussian (no culling)."""
    lights = _c32(lights).reshape(-1, 3)
    radii = _c32(radii)
    L, K = lights.shape[0], radii.shape[0]
    assert K <= 512
    out = np.zeros((L, K, H, W))
    lib().orc_build_tau(_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), sc.n,
                        _pf(lights), L, H, W, _pf(radii), K, float(kappa), _pd(out))
    return out


def build_atlas(sc, lights, H, W, radii, kappa=1.0) -> np.ndarray:
    """Eq. 4: T = exp(-tau), FP64, [L][K][H][W]."""
    return np.exp(-build_tau(sc, lights, H, W, radii, kappa))


def build_tau_texels(sc, lights, H, W, radii, lij, kappa=1.0) -> np.ndarray:
    """tau at the texels lij = [(l,i,j), ...] for all shells: (n, K)."""
    lights = _c32(lights).reshape(-1, 3)
    radii = _c32(radii)
    lij = np.ascontiguousarray(lij, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((lij.shape[0], radii.shape[0]))
    lib().orc_build_tau_texels(_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), sc.n,
                               _pf(lights), H, W, _pf(radii), radii.shape[0], float(kappa),
                               lij.ctypes.data_as(_i32), lij.shape[0], _pd(out))
    return out


def tau_rays(sc, origins, dirs, t, kappa=1.0) -> np.ndarray:
    origins = _c64(origins).reshape(-1, 3)
    dirs = _c64(dirs).reshape(-1, 3)
    t = _c64(t).ravel()
    out = np.zeros(t.shape[0])
    lib().orc_tau_rays(_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), sc.n,
                       _pd(origins), _pd(dirs), _pd(t), t.shape[0], float(kappa), _pd(out))
    return out


# --- sampling / attenuation (Sec. 3.3) ---------------------------------------

def sample_T(atlas_l, radii, o, x) -> float:
    atlas_l = _c64(atlas_l)
    K, H, W = atlas_l.shape
    return float(lib().orc_sample_T(_pd(atlas_l), H, W, _pf(_c32(radii)), K, _pd(_c64(o)),
                                    _pd(_c64(x))))


def attenuate(atlas, radii, lights, q_means, colors, atlas_dyn=None, light_w=None,
              direct_frac=1.0, want_T=False):
    atlas = _c64(atlas)
    L, K, H, W = atlas.shape
    q_means = _c32(q_means)
    colors = _c32(colors)
    Q = q_means.shape[0]
    out = np.zeros((Q, 3))
    T = np.zeros((Q, L)) if want_T else None
    dyn = _c64(atlas_dyn) if atlas_dyn is not None else None
    lw = _c32(light_w) if light_w is not None else None
    lib().orc_attenuate(_pd(atlas), _pd(dyn), L, H, W, _pf(_c32(radii)), K, _pf(_c32(lights)),
                        _pf(q_means), _pf(colors), Q, _pf(lw), float(direct_frac), _pd(out), _pd(T))
    return (out, T) if want_T else out


FOOTPRINT_MODES = {"centre": 0, "stencil7": 1, "mc": 2}


def philox4x64(counter, key) -> np.ndarray:
    """Philox4x64-10 of one counter (4 x uint64) and key (2 x uint64)."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    u64 = C.POINTER(C.c_uint64)
    lib().orc_philox4x64(c.ctypes.data_as(u64), k.ctypes.data_as(u64), out.ctypes.data_as(u64))
    return out


def fp_normal(seed: int, q: int, j: int) -> float:
    """Standard normal number j of receiver q (footprint Monte Carlo offsets)."""
    return float(lib().orc_fp_normal(seed, q, j))


def fp_offsets(mode: str, n_samples: int = 8, seed: int = 0, q: int = 0):
    """(z (n,3), w (n,)) of one receiver's footprint samples."""
    z = np.zeros((64, 3))
    w = np.zeros(64)
    n = lib().orc_fp_offsets(FOOTPRINT_MODES[mode], n_samples, seed, q, _pd(z), _pd(w))
    return z[:n].copy(), w[:n].copy()


def attenuate_footprint(atlas, radii, lights, q_means, q_quats, q_scales, colors, mode="mc",
                        n_samples=8, seed=0, light_w=None, direct_frac=1.0, want_T=False,
                        q_ids=None):
    """Footprint attenuation: T = sum_i w_i T(mu + R (s . z_i)) (Sec. 3.3, ablation (A)).
    q_ids: receiver indices keying the Monte Carlo offsets of each row (default 0..Q-1)."""
    if not 1 <= n_samples <= 64:
        raise ValueError("n_samples must be in 1..64")
    atlas = _c64(atlas)
    L, K, H, W = atlas.shape
    q_means, q_quats, q_scales, colors = (_c32(a) for a in (q_means, q_quats, q_scales, colors))
    Q = q_means.shape[0]
    out = np.zeros((Q, 3))
    T = np.zeros((Q, L)) if want_T else None
    lw = _c32(light_w) if light_w is not None else None
    ids = np.ascontiguousarray(q_ids, dtype=np.int64) if q_ids is not None else None
    if ids is not None and ids.shape != (Q,):
        raise ValueError("q_ids must have one index per receiver")
    lib().orc_attenuate_footprint(_pd(atlas), L, H, W, _pf(_c32(radii)), K, _pf(_c32(lights)),
                                  _pf(q_means), _pf(q_quats), _pf(q_scales), _pf(colors), Q, _pf(lw),
                                  float(direct_frac), FOOTPRINT_MODES[mode], n_samples, seed,
                                  ids.ctypes.data_as(C.POINTER(C.c_int64)) if ids is not None else None,
                                  _pd(out), _pd(T))
    return (out, T) if want_T else out


# --- receiver-driven region of interest (Sec. 3.2) ---------------------------

def roi_box(avatar_means, avatar_opac, R=2.0, z_margin=0.1) -> np.ndarray:
    """(c_x, c_y, R, z_min, z_max): alpha-weighted centroid (x, y) of the avatar
    and the height range of its centres padded by z_margin (FP64)."""
    m = np.asarray(avatar_means, dtype=np.float64)
    a = np.asarray(avatar_opac, dtype=np.float64)
    c = (a[:, None] * m[:, :2]).sum(0) / a.sum()
    return np.array([c[0], c[1], R, m[:, 2].min() - z_margin, m[:, 2].max() + z_margin])


def f32_roi(recv_means, box, lights, H, W, radii):
    """Region of interest: texel mask (L,H,W) uint8 and shell ranges (L,2) int32."""
    recv = _c32(recv_means).reshape(-1, 3)
    lights = _c32(lights).reshape(-1, 3)
    radii = _c32(radii)
    L = lights.shape[0]
    mask = np.zeros((L, H, W), dtype=np.uint8)
    kr = np.zeros((L, 2), dtype=np.int32)
    lib().orc_f32_roi(_pf(recv), recv.shape[0], _pf(_c32(box)), _pf(lights), L, H, W, _pf(radii),
                      radii.shape[0], mask.ctypes.data_as(C.POINTER(C.c_uint8)), kr.ctypes.data_as(_i32))
    return mask, kr


def roi_atlas(atlas, mask, krange) -> np.ndarray:
    """The region-of-interest atlas: the dense atlas on P x [k_min, k_max], 1 elsewhere."""
    out = np.ones_like(atlas)
    L, K = atlas.shape[:2]
    for l in range(L):
        k0, k1 = int(krange[l, 0]), int(krange[l, 1])
        if k1 < k0:
            continue
        sel = mask[l].astype(bool)
        out[l, k0:k1 + 1][:, sel] = atlas[l, k0:k1 + 1][:, sel]
    return out


# --- cubemap probe render (Sec. 3.4) ------------------------------------------

def render_pixels(sc, centre, face, pix, near=0.05) -> np.ndarray:
    """Radiance (len(pix), 3) of probe pixels pix (index f face^2 + i face + j),
    brute force over every Gaussian of sc."""
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    out = np.zeros((pix.shape[0], 3))
    lib().orc_render_pixels(_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), _pf(sc.colors),
                            sc.n, _pf(_c32(centre)), int(face), float(near),
                            pix.ctypes.data_as(C.POINTER(C.c_int64)), pix.shape[0], _pd(out))
    return out


def render_view_pixels(sc, cams, W, H, pix, near=0.05) -> np.ndarray:
    """Radiance (len(pix), 3) of pixels pix (index (v H + i) W + j) of the
    pinhole cameras cams (n_views, 16), brute force over every Gaussian."""
    cams = _c32(cams).reshape(-1, 16)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    out = np.zeros((pix.shape[0], 3))
    lib().orc_render_view_pixels(_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), _pf(sc.colors),
                                 sc.n, _pf(cams), cams.shape[0], int(W), int(H), float(near),
                                 pix.ctypes.data_as(C.POINTER(C.c_int64)), pix.shape[0], _pd(out))
    return out


def cube_cams(centre, face: int) -> np.ndarray:
    """The six probe cameras (6, 16) at centre."""
    out = np.zeros((6, 16), dtype=np.float32)
    lib().orc_cube_cams(_pf(_c32(centre)), int(face), _pf(out))
    return out


def cube_dirs(face: int):
    """Texel-centre unit directions (6 face^2, 3) of the probe, faces
    (+x, -x, +y, -y, +z, -z) with the cube-map axes, rows v, columns u."""
    c = (2.0 * np.arange(face) + 1.0) / face - 1.0
    uu, vv = np.meshgrid(c, c, indexing="xy")
    one = np.ones_like(uu)
    faces = [(one, -vv, -uu), (-one, -vv, uu), (uu, one, vv), (uu, -one, -vv), (uu, -vv, one),
             (-uu, -vv, -one)]
    D = np.concatenate([np.stack(f, -1).reshape(-1, 3) for f in faces])
    return D / np.linalg.norm(D, axis=1, keepdims=True)


# --- FP32 index and binning specification -----------------------------------

def f32_sample_index(points, light, H, W, radii):
    """(ints (n,5): cell i, cell j, base i0, base j0, shell k; floats (n,3): fy, fx, t)."""
    points = _c32(points).reshape(-1, 3)
    n = points.shape[0]
    oi = np.zeros((n, 5), dtype=np.int32)
    of = np.zeros((n, 3), dtype=np.float32)
    radii = _c32(radii)
    lib().orc_f32_sample_index_batch(_pf(points), n, _pf(_c32(light)), H, W, _pf(radii),
                                     radii.shape[0], oi.ctypes.data_as(_i32), _pf(of))
    return oi, of


def f32_rect_cone(i0, i1, j0, j1, H, W) -> np.ndarray:
    out = np.zeros(6, dtype=np.float32)
    lib().orc_f32_rect_cone(i0, i1, j0, j1, H, W, _pf(out))
    return out


def f32_gauss_cone(mu, s, alpha, o, kappa, eps, r_last):
    out = np.zeros(9, dtype=np.float32)
    r = lib().orc_f32_gauss_cone(_pf(_c32(mu)), _pf(_c32(s)), float(alpha), _pf(_c32(o)),
                                 float(kappa), float(eps), float(r_last), _pf(out))
    return r, out


def f32_rect_planes(i0, i1, j0, j1, half, H, W) -> np.ndarray:
    out = np.zeros(17, dtype=np.float32)
    lib().orc_f32_rect_planes(i0, i1, j0, j1, half, H, W, _pf(out))
    return out


def f32_gauss_axes(mu, s, q, o) -> np.ndarray:
    out = np.zeros(12, dtype=np.float32)
    lib().orc_f32_gauss_axes(_pf(_c32(mu)), _pf(_c32(s)), _pf(_c32(q)), _pf(_c32(o)), _pf(out))
    return out


def f32_bin(sc, lights, H, W, radii, kappa=1.0, eps=1e-7, tile=8):
    """Sorted (key, value) pairs of the binning specification; value =
    Gaussian index | half-tile mask << 30."""
    lights = _c32(lights).reshape(-1, 3)
    radii = _c32(radii)
    args = (_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), sc.n, _pf(lights), lights.shape[0],
            H, W, _pf(radii), radii.shape[0], float(kappa), float(eps), int(tile))
    empty = np.zeros(1, dtype=np.uint32)
    total = lib().orc_f32_bin(*args, empty.ctypes.data_as(_u32), empty.ctypes.data_as(_u32), 0)
    if total < 0:
        raise ValueError("invalid Gaussian input")
    keys = np.zeros(max(total, 1), dtype=np.uint32)
    vals = np.zeros(max(total, 1), dtype=np.uint32)
    lib().orc_f32_bin(*args, keys.ctypes.data_as(_u32), vals.ctypes.data_as(_u32), total)
    return keys[:total], vals[:total]


def f32_bin_keys(sc, lights, H, W, radii, keys_wanted, kappa=1.0, eps=1e-7, tile=8):
    """f32_bin restricted to the (light, tile) keys `keys_wanted` (key = l *
    n_tiles + tile): the same (key, value) pairs, only for those tiles."""
    lights = _c32(lights).reshape(-1, 3)
    radii = _c32(radii)
    want = np.unique(np.asarray(keys_wanted, dtype=np.uint32))
    args = (_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac), sc.n, _pf(lights), lights.shape[0],
            H, W, _pf(radii), radii.shape[0], float(kappa), float(eps), int(tile),
            want.ctypes.data_as(_u32), int(want.size))
    empty = np.zeros(1, dtype=np.uint32)
    total = lib().orc_f32_bin_keys(*args, empty.ctypes.data_as(_u32), empty.ctypes.data_as(_u32), 0)
    if total < 0:
        raise ValueError("invalid Gaussian input")
    keys = np.zeros(max(total, 1), dtype=np.uint32)
    vals = np.zeros(max(total, 1), dtype=np.uint32)
    lib().orc_f32_bin_keys(*args, keys.ctypes.data_as(_u32), vals.ctypes.data_as(_u32), total)
    return keys[:total], vals[:total]


def count_ray_evals(sc, lights, H, W, radii, lij, kappa=1.0, eps=1e-7) -> int:
    """Gaussian-ray evaluations the method must make at texels lij (metric units)."""
    lights = _c32(lights).reshape(-1, 3)
    radii = _c32(radii)
    lij = np.ascontiguousarray(lij, dtype=np.int32).reshape(-1, 3)
    return int(lib().orc_count_ray_evals(_pf(sc.means), _pf(sc.scales), _pf(sc.quats), _pf(sc.opac),
                                         sc.n, _pf(lights), H, W, _pf(radii), radii.shape[0],
                                         float(kappa), float(eps), lij.ctypes.data_as(_i32),
                                         lij.shape[0]))


# --- HDRI probe and transfer (Secs. 3.4-3.5) ---------------------------------

def sh_basis(d) -> np.ndarray:
    Y = np.zeros(9)
    lib().orc_sh_basis(_pd(_c64(d)), _pd(Y))
    return Y


def sh_fit(dirs, rgb, w, lam=1e-3) -> np.ndarray:
    """Eq. 7 ridge fit; returns SH (3, 9)."""
    dirs, rgb, w = _c32(dirs), _c32(rgb), _c32(w)
    out = np.zeros(27)
    rc = lib().orc_sh_fit(_pf(dirs), _pf(rgb), _pf(w), dirs.shape[0], float(lam), _pd(out))
    if rc != 0:
        raise np.linalg.LinAlgError("normal equations not positive definite")
    return out.reshape(3, 9)


def gauss_normal(mu, s, q, centroid) -> np.ndarray:
    n = np.zeros(3)
    lib().orc_gauss_normal(_pf(_c32(mu)), _pf(_c32(s)), _pf(_c32(q)), _pf(_c32(centroid)), _pd(n))
    return n


def transfer_scale(sh, n, q=1.0, t_max=10.0, eps=1e-8, n_theta=32, n_phi=64) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_transfer_scale(_pd(_c64(sh)), _pd(_c64(n)), float(q), float(t_max), float(eps),
                             n_theta, n_phi, _pd(out))
    return out


def relight(sh, sc, centroid, normals=None, q=1.0, gamma=1.0, t_max=10.0, eps=1e-8,
            n_theta=32, n_phi=64) -> np.ndarray:
    out = np.zeros((sc.n, 3))
    nrm = _c32(normals) if normals is not None else None
    lib().orc_relight(_pd(_c64(sh)), _pf(sc.means), _pf(sc.quats), _pf(sc.scales), _pf(nrm),
                      _pf(_c32(centroid)), _pf(sc.colors), sc.n, float(q), float(gamma),
                      float(t_max), float(eps), n_theta, n_phi, _pd(out))
    return out
