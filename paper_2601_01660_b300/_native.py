"""ctypes binding of libdgsm.so (include/dgsm.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Tensors must be CUDA, C-contiguous and of the dtype the C ABI
names; results are written into caller-provided or freshly allocated torch
tensors (torch only provides device memory and streams).  If the library is
missing this module raises ImportError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgsm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2601_01660_b300.build`")

_lib = C.CDLL(LIB_PATH)

DGSM_OK = 0
STATUS = {0: "DGSM_OK", 1: "DGSM_ERR_INVALID_ARG", 2: "DGSM_ERR_CUDA", 3: "DGSM_ERR_WORKSPACE",
          4: "DGSM_ERR_TIMEOUT", 5: "DGSM_ERR_NONFINITE_INPUT", 6: "DGSM_ERR_NOT_SPD"}
DTYPES = {"f32": 0, "f16": 1, "bf16": 2}
TORCH_DTYPES = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}


class DGSMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    """Mirror of dgsm_params."""
    _fields_ = [("kappa", C.c_float), ("eps_cull", C.c_float), ("tile", C.c_int32),
                ("chunk", C.c_int32), ("atlas_dtype", C.c_int32), ("max_pairs", C.c_int32),
                ("beta_mode", C.c_int32), ("atlas_map", C.c_int32)]

    @classmethod
    def make(cls, kappa=1.0, eps_cull=1e-7, tile=8, chunk=128, atlas_dtype="f32", max_pairs=0,
             beta_mode=2, atlas_map=0):
        p = cls()
        _lib.dgsm_default_params(C.byref(p))
        p.kappa, p.eps_cull, p.tile, p.chunk, p.max_pairs = kappa, eps_cull, tile, chunk, max_pairs
        p.beta_mode, p.atlas_map = beta_mode, {"octa": 0, "cube": 1}.get(atlas_map, atlas_map)
        p.atlas_dtype = DTYPES[atlas_dtype] if isinstance(atlas_dtype, str) else int(atlas_dtype)
        return p


class Roi(C.Structure):
    """Mirror of dgsm_roi."""
    _fields_ = [("recv_means", C.c_void_p), ("n_recv", C.c_int64), ("box", C.c_void_p),
                ("mask_out", C.c_void_p), ("krange_out", C.c_void_p)]


class RelightParams(C.Structure):
    """Mirror of dgsm_relight_params."""
    _fields_ = [("q", C.c_float), ("gamma", C.c_float), ("t_max", C.c_float), ("eps", C.c_float),
                ("n_theta", C.c_int32), ("n_phi", C.c_int32)]

    @classmethod
    def make(cls, q=1.0, gamma=1.0, t_max=10.0, eps=1e-8, n_theta=32, n_phi=64):
        p = cls()
        p.q, p.gamma, p.t_max, p.eps, p.n_theta, p.n_phi = q, gamma, t_max, eps, n_theta, n_phi
        return p


class BuildStats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("rays_tested", C.c_int64), ("ray_evals", C.c_int64),
                ("shell_evals", C.c_int64), ("n_super_pairs", C.c_int64)]


class FrameHostIn(C.Structure):
    """Mirror of dgsm_frame_host_in (host pointers)."""
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p),
                ("opac", C.c_void_p), ("colors", C.c_void_p), ("n", C.c_int64),
                ("relight_begin", C.c_int64), ("relight_end", C.c_int64), ("lights", C.c_void_p),
                ("n_lights", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("K", C.c_int32),
                ("radii", C.c_void_p), ("cube_dirs", C.c_void_p), ("cube_rgb", C.c_void_p),
                ("cube_w", C.c_void_p), ("n_cube", C.c_int64), ("lam", C.c_double)]


class CrowdFrameArgs(C.Structure):
    """Mirror of dgsm_crowd_frame_args (device pointers except seg, and poses when pinned)."""
    _fields_ = [("q_means", C.c_void_p), ("colors_in", C.c_void_p), ("colors_out", C.c_void_p),
                ("n_static", C.c_int64), ("static_atlas", C.c_void_p), ("H", C.c_int32), ("W", C.c_int32),
                ("K", C.c_int32), ("radii", C.c_void_p), ("rest_means", C.c_void_p), ("rest_quats", C.c_void_p),
                ("scales", C.c_void_p), ("opac", C.c_void_p), ("quats_out", C.c_void_p), ("n_avatar", C.c_int64),
                ("seg", C.c_void_p), ("n_obj", C.c_int32), ("poses", C.c_void_p), ("dyn_atlas", C.c_void_p),
                ("H_dyn", C.c_int32), ("W_dyn", C.c_int32), ("K_dyn", C.c_int32), ("radii_dyn", C.c_void_p),
                ("lights", C.c_void_p), ("L", C.c_int32), ("sh", C.c_void_p), ("centroids_out", C.c_void_p),
                ("direct_frac", C.c_float)]


_vp = C.c_void_p
_i32, _i64, _f32, _f64 = C.c_int32, C.c_int64, C.c_float, C.c_double

_lib.dgsm_default_params.argtypes = [C.POINTER(Params)]
_lib.dgsm_default_relight_params.argtypes = [C.POINTER(RelightParams)]
_lib.dgsm_create.argtypes = [C.c_int, C.POINTER(_vp)]
_lib.dgsm_create.restype = C.c_int
_lib.dgsm_destroy.argtypes = [_vp]
_lib.dgsm_last_error.argtypes = [_vp]
_lib.dgsm_last_error.restype = C.c_char_p
_lib.dgsm_status_string.argtypes = [C.c_int]
_lib.dgsm_status_string.restype = C.c_char_p
_lib.dgsm_build.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _i32,
                            C.POINTER(Params), _vp, _vp]
_lib.dgsm_get_build_stats.argtypes = [_vp, C.POINTER(BuildStats)]
_lib.dgsm_build_roi.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _i32,
                                C.POINTER(Params), C.POINTER(Roi), _vp, _vp]
_lib.dgsm_roi_box.argtypes = [_vp, _vp, _vp, _i64, _f32, _f32, _vp, _vp]
_lib.dgsm_build_band.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _i32,
                                 C.POINTER(Params), _i32, _i32, _vp, _vp]
_lib.dgsm_atlas_rows_copy.argtypes = [_vp, _vp, _i32, _i32, _vp, _i32, _i32, _i32, _i64, _i32, _i32, _vp]
_lib.dgsm_pca_normals.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _f32, _vp, _vp, _vp]
_lib.dgsm_spatial_order.argtypes = [_vp, _vp, _i64, _vp, _vp]
_lib.dgsm_gather_rows.argtypes = [_vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp]
_lib.dgsm_bin.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _i32,
                          C.POINTER(Params), _vp, _vp, _i64, C.POINTER(_i64), _vp]
_lib.dgsm_attenuate.argtypes = [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp,
                                _i64, _vp, _f32, _vp, _vp, _vp]
_lib.dgsm_attenuate_dyn.argtypes = [_vp, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _i32, _i32, _vp,
                                    _i32, _vp, _vp, _vp, _i64, _vp, _f32, _vp, _vp, _vp]
_lib.dgsm_sample_index.argtypes = [_vp, _vp, _i64, _vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp]
_lib.dgsm_attenuate_cube.argtypes = [_vp, _vp, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _i64, _vp, _f32,
                                     _vp, _vp, _vp]
_lib.dgsm_sample_index_cube.argtypes = [_vp, _vp, _i64, _vp, _i32, _vp, _i32, _vp, _vp, _vp]
_lib.dgsm_attenuate_footprint.argtypes = [_vp, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp,
                                          _vp, _vp, _i64, _vp, _f32, _i32, _i32, C.c_uint64, _vp,
                                          _vp, _vp]
_lib.sh_fit.argtypes = [_vp, _vp, _vp, _vp, _i64, _f64, _vp, _vp, _vp]
_lib.dgsm_render_cubemap.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _f32, _vp,
                                     C.POINTER(_i64), _vp]
_lib.dgsm_cube_dirs.argtypes = [_vp, _i32, _vp, _vp, _vp]
_lib.dgsm_render_views.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _f32, _vp,
                                   C.POINTER(_i64), _vp]
_lib.sh_fit_static.argtypes = [_vp, _vp, _vp, _i64, _f64, _vp, _vp, _vp, _vp]
_lib.sh_relight.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64,
                            C.POINTER(RelightParams), _vp, _vp]
_lib.dgsm_sync_status.argtypes = [_vp, _vp]
_lib.dgsm_selftest_wait.argtypes = [_vp, _i32, _i64, _vp]
_lib.dgsm_weighted_centroid.argtypes = [_vp, _vp, _vp, _i64, _vp, _vp]
_lib.dgsm_frame_host.argtypes = [_vp, C.POINTER(FrameHostIn), C.POINTER(Params),
                                 C.POINTER(RelightParams), _vp, _vp, _vp]
_lib.dgsm_frame_host_submit.argtypes = [_vp, _i32, C.POINTER(FrameHostIn), C.POINTER(Params),
                                       C.POINTER(RelightParams), _vp, _vp, _vp]
_lib.dgsm_frame_host_wait.argtypes = [_vp, _i32]
_lib.nf_param_count.restype = C.c_int64
_lib.nf_param_count.argtypes = []
_lib.nf_init.argtypes = [_vp, C.c_uint64, _vp, _vp]
_lib.nf_loss_grad.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]
_lib.nf_train.argtypes = [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _i32, _i32, _f32, C.c_uint64,
                          _i32, _vp, _vp]
_lib.nf_forward.argtypes = [_vp, _vp, _vp, _i64, _vp, _vp]
_lib.nf_tile_error.argtypes = [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp]
_lib.nf_attenuate.argtypes = [_vp, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _i32, _i32, _vp, _vp, _vp,
                              _i64, _vp, _f32, _vp, _vp, _vp]
_lib.sh_relight_objects.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _i64,
                                    C.POINTER(RelightParams), _vp, _vp]
_lib.dgsm_segment_centroids.argtypes = [_vp, _vp, _vp, _i64, _vp, _i32, _vp, _vp]
_lib.dgsm_rigid_transform.argtypes = [_vp, _vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp, _vp]
_lib.dgsm_crowd_frame.argtypes = [_vp, C.POINTER(CrowdFrameArgs), C.POINTER(Params), C.POINTER(RelightParams),
                                  _i32, _vp]
_lib.dgsm_crowd_frame_phases.argtypes = [_vp, C.POINTER(C.c_double)]
_lib.dgsm_graph_begin.argtypes = [_vp, _vp]
_lib.dgsm_graph_end.argtypes = [_vp, _vp, C.POINTER(_vp)]
_lib.dgsm_graph_launch.argtypes = [_vp, _vp]
_lib.dgsm_graph_node_count.argtypes = [_vp, C.POINTER(_i64)]
_lib.dgsm_graph_destroy.argtypes = [_vp]
_lib.dgsm_graph_destroy.restype = None
_lib.dgsm_autotune_build.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _i32,
                                     C.POINTER(Params), _vp, _i32, _vp, _i32, _i32, _vp,
                                     C.POINTER(Params), _vp, _vp]
_lib.dgsm_set_profiling.argtypes = [_vp, C.c_int]
_lib.dgsm_measure_alu_peaks.argtypes = [_vp, C.POINTER(C.c_double), _vp]
_lib.dgsm_profile_collect.argtypes = [_vp, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]
for _fn in ("dgsm_build", "dgsm_get_build_stats", "dgsm_bin", "dgsm_attenuate",
            "dgsm_sample_index", "sh_fit", "sh_relight", "dgsm_sync_status",
            "dgsm_weighted_centroid", "dgsm_frame_host", "dgsm_set_profiling",
            "dgsm_profile_collect", "sh_fit_static", "nf_init", "nf_loss_grad", "nf_train", "nf_forward",
            "nf_tile_error", "nf_attenuate", "sh_relight_objects", "dgsm_segment_centroids",
            "dgsm_rigid_transform", "dgsm_graph_begin", "dgsm_graph_end", "dgsm_graph_launch",
            "dgsm_graph_node_count", "dgsm_autotune_build", "dgsm_attenuate_dyn",
            "dgsm_measure_alu_peaks", "dgsm_frame_host_submit", "dgsm_frame_host_wait",
            "dgsm_spatial_order", "dgsm_gather_rows"):
    getattr(_lib, _fn).restype = C.c_int


class Context:
    """Owns a dgsm_ctx (device workspace, status word) on one device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = _vp()
        rc = _lib.dgsm_create(self.device, C.byref(h))
        if rc != DGSM_OK:
            raise DGSMError(rc, "dgsm_create failed")
        self._h = h

    @property
    def handle(self):
        return self._h

    def check(self, rc: int):
        if rc != DGSM_OK:
            raise DGSMError(rc, _lib.dgsm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.dgsm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ctx_lock = threading.Lock()
_contexts: dict[int, Context] = {}


def context(device: int | None = None) -> Context:
    """The process-wide default context of `device` (current device if None)."""
    if device is None:
        device = torch.cuda.current_device()
    with _ctx_lock:
        if device not in _contexts:
            _contexts[device] = Context(device)
        return _contexts[device]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(t, name, dtype=torch.float32, shape_last=None):
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"{name} must have shape (n, {shape_last})")
    return t


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def dgsm_build(means, scales, quats, opac, lights, H, W, radii, params=None, out=None,
               ctx: Context | None = None, stream=None):
    """Deep Gaussian Shadow Map build (Sec. 3.2): returns the atlas [L][K][H][W]."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    _need(scales, "scales", shape_last=3)
    _need(quats, "quats", shape_last=4)
    _need(opac, "opac")
    _need(lights, "lights", shape_last=3)
    _need(radii, "radii")
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    L, K, n = lights.shape[0], radii.shape[0], means.shape[0]
    if out is None:
        out = torch.empty((L, K, H, W), dtype=TORCH_DTYPES[p.atlas_dtype], device=means.device)
    _need(out, "out", TORCH_DTYPES[p.atlas_dtype])
    if tuple(out.shape) != (L, K, H, W):
        raise ValueError("out must have shape (L, K, H, W)")
    ctx.check(_lib.dgsm_build(ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac), n,
                              _ptr(lights), L, H, W, _ptr(radii), K, C.byref(p), _ptr(out),
                              _stream(stream)))
    return out


def dgsm_build_band(means, scales, quats, opac, lights, H, W, radii, row0, row1, params=None, out=None,
                    ctx: Context | None = None, stream=None):
    """Rows [row0, row1) of the atlas [L][K][H][W] as dgsm_build builds them,
    T = 1 elsewhere (one GPU's band of a light's atlas)."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    _need(scales, "scales", shape_last=3)
    _need(quats, "quats", shape_last=4)
    _need(opac, "opac")
    _need(lights, "lights", shape_last=3)
    _need(radii, "radii")
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    L, K, n = lights.shape[0], radii.shape[0], means.shape[0]
    if out is None:
        out = torch.empty((L, K, H, W), dtype=TORCH_DTYPES[p.atlas_dtype], device=means.device)
    _need(out, "out", TORCH_DTYPES[p.atlas_dtype])
    if tuple(out.shape) != (L, K, H, W):
        raise ValueError("out must have shape (L, K, H, W)")
    ctx.check(_lib.dgsm_build_band(ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac), n,
                                   _ptr(lights), L, H, W, _ptr(radii), K, C.byref(p), int(row0), int(row1),
                                   _ptr(out), _stream(stream)))
    return out


def dgsm_atlas_rows_copy(src, src_row0, dst, dst_row0, rows, ctx: Context | None = None, stream=None):
    """dst[..., dst_row0:dst_row0+rows, :] = src[..., src_row0:src_row0+rows, :] for
    contiguous (..., rows, W) device tensors of one dtype and the same leading shape."""
    ctx = ctx or context(src.device.index)
    _need(src, "src", src.dtype)
    _need(dst, "dst", src.dtype)
    if src.dim() < 2 or src.shape[:-2] != dst.shape[:-2] or src.shape[-1] != dst.shape[-1]:
        raise ValueError("src and dst must share their leading shape and width")
    planes = 1
    for d in src.shape[:-2]:
        planes *= int(d)
    ctx.check(_lib.dgsm_atlas_rows_copy(ctx.handle, _ptr(src), src.shape[-2], int(src_row0), _ptr(dst),
                                        dst.shape[-2], int(dst_row0), int(rows), planes, src.shape[-1],
                                        src.element_size(), _stream(stream)))
    return dst


def dgsm_get_build_stats(ctx: Context | None = None) -> dict:
    ctx = ctx or context()
    st = BuildStats()
    ctx.check(_lib.dgsm_get_build_stats(ctx.handle, C.byref(st)))
    return {"n_pairs": st.n_pairs, "rays_tested": st.rays_tested, "ray_evals": st.ray_evals,
            "shell_evals": st.shell_evals, "n_super_pairs": st.n_super_pairs}


def dgsm_bin(means, scales, quats, opac, lights, H, W, radii, params=None, ctx: Context | None = None,
             stream=None):
    """Light-space tile binning: sorted (keys, values) int32 tensors holding the
    uint32 key and value (Gaussian index | half-tile mask << 30)."""
    ctx = ctx or context(means.device.index)
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    L, K, n = lights.shape[0], radii.shape[0], means.shape[0]
    total = _i64(0)
    args = (ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac), n, _ptr(lights), L, H, W,
            _ptr(radii), K, C.byref(p))
    rc = _lib.dgsm_bin(*args, None, None, 0, C.byref(total), _stream(stream))
    if rc not in (DGSM_OK, 3):
        ctx.check(rc)
    P = total.value
    keys = torch.empty(max(P, 1), dtype=torch.int32, device=means.device)
    vals = torch.empty(max(P, 1), dtype=torch.int32, device=means.device)
    ctx.check(_lib.dgsm_bin(*args, _ptr(keys), _ptr(vals), P, C.byref(total), _stream(stream)))
    return keys[:P], vals[:P]


def dgsm_build_roi(means, scales, quats, opac, lights, H, W, radii, recv_means, box, params=None,
                   out=None, want_roi=False, ctx: Context | None = None, stream=None):
    """dgsm_build on a receiver-driven region of interest (Sec. 3.2): the atlas
    equals the dense one on P x [k_min, k_max] and is 1 elsewhere.  box: device
    (5,) float32 (c_x, c_y, R, z_min, z_max).  With want_roi also returns the
    texel mask (L, H, W) uint8 and the shell ranges (L, 2) int32."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    _need(scales, "scales", shape_last=3)
    _need(quats, "quats", shape_last=4)
    _need(opac, "opac")
    _need(lights, "lights", shape_last=3)
    _need(radii, "radii")
    _need(recv_means, "recv_means", shape_last=3)
    _need(box, "box")
    if box.numel() != 5:
        raise ValueError("box must hold 5 floats")
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    L, K, n = lights.shape[0], radii.shape[0], means.shape[0]
    if out is None:
        out = torch.empty((L, K, H, W), dtype=TORCH_DTYPES[p.atlas_dtype], device=means.device)
    _need(out, "out", TORCH_DTYPES[p.atlas_dtype])
    if tuple(out.shape) != (L, K, H, W):
        raise ValueError("out must have shape (L, K, H, W)")
    mask = torch.empty((L, H, W), dtype=torch.uint8, device=means.device) if want_roi else None
    kr = torch.empty((L, 2), dtype=torch.int32, device=means.device) if want_roi else None
    addr = lambda t: None if t is None else t.data_ptr()
    roi = Roi(addr(recv_means), recv_means.shape[0], addr(box), addr(mask), addr(kr))
    ctx.check(_lib.dgsm_build_roi(ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac), n,
                                  _ptr(lights), L, H, W, _ptr(radii), K, C.byref(p), C.byref(roi),
                                  _ptr(out), _stream(stream)))
    return (out, mask, kr) if want_roi else out


def dgsm_roi_box(avatar_means, avatar_opac, R=2.0, z_margin=0.1, out=None,
                 ctx: Context | None = None, stream=None):
    """Box (c_x, c_y, R, z_min, z_max) around an avatar: alpha-weighted centroid
    and padded height range of its centres (Sec. 3.2)."""
    ctx = ctx or context(avatar_means.device.index)
    _need(avatar_means, "avatar_means", shape_last=3)
    _need(avatar_opac, "avatar_opac")
    if out is None:
        out = torch.empty(5, dtype=torch.float32, device=avatar_means.device)
    ctx.check(_lib.dgsm_roi_box(ctx.handle, _ptr(avatar_means), _ptr(avatar_opac), avatar_means.shape[0],
                                float(R), float(z_margin), _ptr(out), _stream(stream)))
    return out


def dgsm_pca_normals(means, opac, quats, scales, centroid, radius=0.05, out=None,
                     ctx: Context | None = None, stream=None):
    """Pseudo-normals (n, 3) by alpha- and distance-weighted local PCA of the
    Gaussian centres within `radius` (Sec. 4), the smallest-scale axis where
    the neighbourhood is too sparse; turned away from `centroid` (device, 3)."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    _need(opac, "opac")
    _need(quats, "quats", shape_last=4)
    _need(scales, "scales", shape_last=3)
    _need(centroid, "centroid")
    n = means.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=means.device)
    ctx.check(_lib.dgsm_pca_normals(ctx.handle, _ptr(means), _ptr(opac), _ptr(quats), _ptr(scales), n,
                                    float(radius), _ptr(centroid), _ptr(out), _stream(stream)))
    return out


def dgsm_spatial_order(means, ctx: Context | None = None, stream=None):
    """The permutation (n int32, device) that puts a scene in the Z-order of
    its means (a storage order: no per-Gaussian result depends on it)."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    n = means.shape[0]
    perm = torch.empty((n,), dtype=torch.int32, device=means.device)
    ctx.check(_lib.dgsm_spatial_order(ctx.handle, _ptr(means), n, _ptr(perm), _stream(stream)))
    return perm


def dgsm_gather_rows(src, perm, out=None, ctx: Context | None = None, stream=None):
    """out[i] = src[perm[i]] over the first dimension (any 4-byte dtype
    layout: rows of a multiple of 4 bytes)."""
    ctx = ctx or context(src.device.index)
    if not src.is_cuda or not src.is_contiguous() or src.dim() < 1:
        raise ValueError("src must be a contiguous CUDA tensor")
    _need(perm, "perm", dtype=torch.int32)
    n = perm.shape[0]
    if out is None:
        out = torch.empty((n,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    if out.shape[1:] != src.shape[1:] or out.dtype != src.dtype or not out.is_contiguous() or out.shape[0] != n:
        raise ValueError("out must be a contiguous tensor of perm's length and src's row shape and dtype")
    row_bytes = math.prod(src.shape[1:]) * src.element_size()
    ctx.check(_lib.dgsm_gather_rows(ctx.handle, _ptr(src), src.shape[0], row_bytes, _ptr(perm), n, _ptr(out),
                                    _stream(stream)))
    return out


def dgsm_render_cubemap(means, scales, quats, opac, colors, centre, face=64, near=0.05, out=None,
                        want_pairs=False, ctx: Context | None = None, stream=None):
    """Cubemap probe (Sec. 3.4): the scene splatted on the six 90-degree faces
    at `centre` (device, 3 floats); returns (6 * face^2, 3) radiance."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    _need(scales, "scales", shape_last=3)
    _need(quats, "quats", shape_last=4)
    _need(opac, "opac")
    _need(colors, "colors", shape_last=3)
    _need(centre, "centre")
    if out is None:
        out = torch.empty((6 * face * face, 3), dtype=torch.float32, device=means.device)
    npairs = _i64(0)
    ctx.check(_lib.dgsm_render_cubemap(ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac),
                                       _ptr(colors), means.shape[0], _ptr(centre), int(face), float(near),
                                       _ptr(out), C.byref(npairs), _stream(stream)))
    return (out, npairs.value) if want_pairs else out


def dgsm_render_views(means, scales, quats, opac, colors, cams, W, H, near=0.05, out=None,
                      want_pairs=False, ctx: Context | None = None, stream=None):
    """3DGS splatting into pinhole cameras: cams (n_views, 16) float32 on the
    device (R row-major rows x, y, forward; position; fx, fy, cx, cy);
    returns (n_views, H, W, 3) radiance."""
    ctx = ctx or context(means.device.index)
    for t, nm, last in ((means, "means", 3), (scales, "scales", 3), (quats, "quats", 4), (colors, "colors", 3)):
        _need(t, nm, shape_last=last)
    _need(opac, "opac")
    _need(cams, "cams", shape_last=16)
    V = cams.shape[0]
    if out is None:
        out = torch.empty((V, H, W, 3), dtype=torch.float32, device=means.device)
    npairs = _i64(0)
    ctx.check(_lib.dgsm_render_views(ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac),
                                     _ptr(colors), means.shape[0], _ptr(cams), V, int(W), int(H), float(near),
                                     _ptr(out), C.byref(npairs), _stream(stream)))
    return (out, npairs.value) if want_pairs else out


def dgsm_cube_dirs(face=64, device=None, ctx: Context | None = None, stream=None):
    """(dirs (6 face^2, 3), solid angles (6 face^2)) of the probe's pixels."""
    ctx = ctx or context(device)
    dev = torch.device("cuda", ctx.device)
    dirs = torch.empty((6 * face * face, 3), dtype=torch.float32, device=dev)
    w = torch.empty(6 * face * face, dtype=torch.float32, device=dev)
    ctx.check(_lib.dgsm_cube_dirs(ctx.handle, int(face), _ptr(dirs), _ptr(w), _stream(stream)))
    return dirs, w


def dgsm_attenuate(atlas, radii, lights, q_means, colors, atlas_dyn=None, light_w=None,
                   direct_frac=1.0, out=None, want_T=False, ctx: Context | None = None,
                   stream=None):
    """Receiver attenuation (Sec. 3.3): colours (and T per light if want_T)."""
    ctx = ctx or context(atlas.device.index)
    dt = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}[atlas.dtype]
    _need(atlas, "atlas", atlas.dtype)
    L, K, H, W = atlas.shape
    _need(radii, "radii")
    _need(lights, "lights", shape_last=3)
    _need(q_means, "q_means", shape_last=3)
    _need(colors, "colors", shape_last=3)
    if atlas_dyn is not None:
        _need(atlas_dyn, "atlas_dyn", atlas.dtype)
        if atlas_dyn.shape != atlas.shape:
            raise ValueError("atlas_dyn must match atlas")
    if light_w is not None:
        _need(light_w, "light_w")
    Q = q_means.shape[0]
    if out is None:
        out = torch.empty_like(colors)
    T = torch.empty((Q, L), dtype=torch.float32, device=atlas.device) if want_T else None
    ctx.check(_lib.dgsm_attenuate(ctx.handle, _ptr(atlas), _ptr(atlas_dyn), dt, L, H, W,
                                  _ptr(radii), K, _ptr(lights), _ptr(q_means), _ptr(colors), Q,
                                  _ptr(light_w), float(direct_frac), _ptr(out), _ptr(T),
                                  _stream(stream)))
    return (out, T) if want_T else out


FOOTPRINT_MODES = {"centre": 0, "stencil7": 1, "mc": 2}


def dgsm_attenuate_footprint(atlas, radii, lights, q_means, q_quats, q_scales, colors, mode="mc",
                             n_samples=8, seed=0, light_w=None, direct_frac=1.0, out=None,
                             want_T=False, ctx: Context | None = None, stream=None):
    """Footprint attenuation (Sec. 3.3; ablation (A)): T averaged over
    x_i = mu + R (s . z_i) with the 7-point stencil or n_samples Monte Carlo
    offsets (Philox4x64-10 keyed by seed and receiver index)."""
    ctx = ctx or context(atlas.device.index)
    dt = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}[atlas.dtype]
    _need(atlas, "atlas", atlas.dtype)
    L, K, H, W = atlas.shape
    _need(radii, "radii")
    _need(lights, "lights", shape_last=3)
    _need(q_means, "q_means", shape_last=3)
    _need(q_quats, "q_quats", shape_last=4)
    _need(q_scales, "q_scales", shape_last=3)
    _need(colors, "colors", shape_last=3)
    if light_w is not None:
        _need(light_w, "light_w")
    Q = q_means.shape[0]
    if out is None:
        out = torch.empty_like(colors)
    T = torch.empty((Q, L), dtype=torch.float32, device=atlas.device) if want_T else None
    ctx.check(_lib.dgsm_attenuate_footprint(
        ctx.handle, _ptr(atlas), dt, L, H, W, _ptr(radii), K, _ptr(lights), _ptr(q_means),
        _ptr(q_quats), _ptr(q_scales), _ptr(colors), Q, _ptr(light_w), float(direct_frac),
        FOOTPRINT_MODES[mode], int(n_samples), int(seed) & (2**64 - 1), _ptr(out), _ptr(T),
        _stream(stream)))
    return (out, T) if want_T else out


def dgsm_attenuate_cube(atlas, radii, lights, q_means, colors, light_w=None, direct_frac=1.0, out=None,
                        want_T=False, ctx: Context | None = None, stream=None):
    """Receiver attenuation through a cube-map atlas [L][K][6F][F] (atlas_map = 1)."""
    ctx = ctx or context(atlas.device.index)
    dt = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}[atlas.dtype]
    _need(atlas, "atlas", atlas.dtype)
    L, K, H, F = atlas.shape
    if H != 6 * F:
        raise ValueError("a cube atlas has H = 6 W")
    _need(radii, "radii")
    _need(lights, "lights", shape_last=3)
    _need(q_means, "q_means", shape_last=3)
    _need(colors, "colors", shape_last=3)
    Q = q_means.shape[0]
    if out is None:
        out = torch.empty_like(colors)
    T = torch.empty((Q, L), dtype=torch.float32, device=atlas.device) if want_T else None
    ctx.check(_lib.dgsm_attenuate_cube(ctx.handle, _ptr(atlas), dt, L, F, _ptr(radii), K, _ptr(lights),
                                       _ptr(q_means), _ptr(colors), Q, _ptr(light_w), float(direct_frac), _ptr(out),
                                       _ptr(T), _stream(stream)))
    return (out, T) if want_T else out


def dgsm_sample_index_cube(points, light, F, radii, ctx: Context | None = None, stream=None):
    """Integer decisions of the cube-map lookup: idx (n,5) int32 (cell row
    (global), cell column, base row (global), base column, shell), frac (n,3)."""
    ctx = ctx or context(points.device.index)
    _need(points, "points", shape_last=3)
    n = points.shape[0]
    idx = torch.empty((n, 5), dtype=torch.int32, device=points.device)
    frac = torch.empty((n, 3), dtype=torch.float32, device=points.device)
    ctx.check(_lib.dgsm_sample_index_cube(ctx.handle, _ptr(points), n, _ptr(light), int(F), _ptr(radii),
                                          radii.shape[0], _ptr(idx), _ptr(frac), _stream(stream)))
    return idx, frac


def dgsm_attenuate_dyn(atlas, radii, atlas_dyn, radii_dyn, lights, q_means, colors, light_w=None,
                       direct_frac=1.0, out=None, want_T=False, ctx: Context | None = None,
                       stream=None):
    """Attenuation by a static atlas times a dynamic atlas of its own shape."""
    ctx = ctx or context(atlas.device.index)
    dt = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}[atlas.dtype]
    _need(atlas, "atlas", atlas.dtype)
    _need(atlas_dyn, "atlas_dyn", atlas.dtype)
    L, K, H, W = atlas.shape
    Ld, Kd, Hd, Wd = atlas_dyn.shape
    if Ld != L:
        raise ValueError("atlas_dyn must have one atlas per light")
    for t, nm in ((radii, "radii"), (radii_dyn, "radii_dyn")):
        _need(t, nm)
    _need(lights, "lights", shape_last=3)
    _need(q_means, "q_means", shape_last=3)
    _need(colors, "colors", shape_last=3)
    if light_w is not None:
        _need(light_w, "light_w")
    Q = q_means.shape[0]
    if out is None:
        out = torch.empty_like(colors)
    T = torch.empty((Q, L), dtype=torch.float32, device=atlas.device) if want_T else None
    ctx.check(_lib.dgsm_attenuate_dyn(ctx.handle, _ptr(atlas), dt, L, H, W, _ptr(radii), K,
                                      _ptr(atlas_dyn), Hd, Wd, _ptr(radii_dyn), Kd, _ptr(lights),
                                      _ptr(q_means), _ptr(colors), Q, _ptr(light_w),
                                      float(direct_frac), _ptr(out), _ptr(T), _stream(stream)))
    return (out, T) if want_T else out


def dgsm_sample_index(points, light, H, W, radii, ctx: Context | None = None, stream=None):
    ctx = ctx or context(points.device.index)
    _need(points, "points", shape_last=3)
    n = points.shape[0]
    idx = torch.empty((n, 5), dtype=torch.int32, device=points.device)
    frac = torch.empty((n, 3), dtype=torch.float32, device=points.device)
    ctx.check(_lib.dgsm_sample_index(ctx.handle, _ptr(points), n, _ptr(light), H, W, _ptr(radii),
                                     radii.shape[0], _ptr(idx), _ptr(frac), _stream(stream)))
    return idx, frac


def sh_fit(dirs, rgb, w, lam=1e-3, want64=False, ctx: Context | None = None, stream=None):
    """HDRI probe fit (Sec. 3.4, Eq. 7) in FP64 on the GPU: SH (3, 9) float32."""
    ctx = ctx or context(dirs.device.index)
    _need(dirs, "dirs", shape_last=3)
    _need(rgb, "rgb", shape_last=3)
    _need(w, "w")
    sh = torch.empty((3, 9), dtype=torch.float32, device=dirs.device)
    sh64 = torch.empty((3, 9), dtype=torch.float64, device=dirs.device) if want64 else None
    ctx.check(_lib.sh_fit(ctx.handle, _ptr(dirs), _ptr(rgb), _ptr(w), dirs.shape[0], float(lam),
                          _ptr(sh), _ptr(sh64), _stream(stream)))
    return (sh, sh64) if want64 else sh


def sh_fit_static(dirs, rgb, w, lam=1e-3, stream=None):
    """sh_fit through the allocation-free entry point: (sh (3,9) float32,
    sh (3,9) float64, status (1,) int32), all on the device.  The output
    tensors here come from torch; the library itself allocates nothing."""
    _need(dirs, "dirs", shape_last=3)
    _need(rgb, "rgb", shape_last=3)
    _need(w, "w")
    sh = torch.empty((3, 9), dtype=torch.float32, device=dirs.device)
    sh64 = torch.empty((3, 9), dtype=torch.float64, device=dirs.device)
    status = torch.empty(1, dtype=torch.int32, device=dirs.device)
    rc = _lib.sh_fit_static(_ptr(dirs), _ptr(rgb), _ptr(w), dirs.shape[0], float(lam), _ptr(sh),
                            _ptr(sh64), _ptr(status), _stream(stream))
    if rc != DGSM_OK:
        raise DGSMError(rc, "sh_fit_static failed")
    return sh, sh64, status


def sh_relight(sh, means, quats, scales, colors, centroid, normals=None, params=None, out=None,
               ctx: Context | None = None, stream=None):
    """Per-Gaussian radiance transfer (Sec. 3.5, Eqs. 8-10): relit colours."""
    ctx = ctx or context(colors.device.index)
    _need(sh, "sh")
    _need(colors, "colors", shape_last=3)
    n = colors.shape[0]
    if normals is None:
        _need(means, "means", shape_last=3)
        _need(quats, "quats", shape_last=4)
        _need(scales, "scales", shape_last=3)
        _need(centroid, "centroid")
    else:
        _need(normals, "normals", shape_last=3)
    p = params if isinstance(params, RelightParams) else RelightParams.make(**(params or {}))
    if out is None:
        out = torch.empty_like(colors)
    ctx.check(_lib.sh_relight(ctx.handle, _ptr(sh), _ptr(means), _ptr(quats), _ptr(scales),
                              _ptr(normals), _ptr(centroid), _ptr(colors), n, C.byref(p), _ptr(out),
                              _stream(stream)))
    return out


def _segs(seg, n):
    seg = [int(x) for x in seg]
    if len(seg) < 2 or seg[0] != 0 or seg[-1] != n:
        raise ValueError("seg must run from 0 to n")
    return (C.c_int64 * len(seg))(*seg), len(seg) - 1


def sh_relight_objects(sh, means, quats, scales, colors, centroids, seg, params=None, out=None,
                       ctx: Context | None = None, stream=None):
    """sh_relight over contiguous objects (object o = Gaussians seg[o]:seg[o+1]),
    each with its own centroid row (n_obj, 3)."""
    ctx = ctx or context(colors.device.index)
    for t, nm, k in ((sh, "sh", None), (means, "means", 3), (quats, "quats", 4), (scales, "scales", 3),
                     (colors, "colors", 3), (centroids, "centroids", 3)):
        _need(t, nm, shape_last=k)
    n = colors.shape[0]
    segs, n_obj = _segs(seg, n)
    p = params if isinstance(params, RelightParams) else RelightParams.make(**(params or {}))
    if out is None:
        out = torch.empty_like(colors)
    ctx.check(_lib.sh_relight_objects(ctx.handle, _ptr(sh), _ptr(means), _ptr(quats), _ptr(scales),
                                      _ptr(centroids), segs, n_obj, _ptr(colors), n, C.byref(p),
                                      _ptr(out), _stream(stream)))
    return out


def dgsm_segment_centroids(means, weights, seg, out=None, ctx: Context | None = None, stream=None):
    """Alpha-weighted centroid of each contiguous object: (n_obj, 3) float32."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    if weights is not None:
        _need(weights, "weights")
    n = means.shape[0]
    segs, n_obj = _segs(seg, n)
    if out is None:
        out = torch.empty((n_obj, 3), dtype=torch.float32, device=means.device)
    ctx.check(_lib.dgsm_segment_centroids(ctx.handle, _ptr(means), _ptr(weights), n, segs, n_obj,
                                          _ptr(out), _stream(stream)))
    return out


def dgsm_rigid_transform(means, quats, seg, poses, means_out=None, quats_out=None,
                         ctx: Context | None = None, stream=None):
    """Rigid motion of contiguous objects; poses (n_obj, 8) float32 =
    (qw, qx, qy, qz, tx, ty, tz, unused), on the device or in (pinned) host memory."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    _need(quats, "quats", shape_last=4)
    if poses.dtype != torch.float32 or not poses.is_contiguous() or tuple(poses.shape[1:]) != (8,):
        raise ValueError("poses must be a contiguous (n_obj, 8) float32 tensor")
    n = means.shape[0]
    segs, n_obj = _segs(seg, n)
    if poses.shape[0] != n_obj:
        raise ValueError("one pose per object")
    means_out = torch.empty_like(means) if means_out is None else means_out
    quats_out = torch.empty_like(quats) if quats_out is None else quats_out
    ctx.check(_lib.dgsm_rigid_transform(ctx.handle, _ptr(means), _ptr(quats), n, segs, n_obj,
                                        _ptr(poses), _ptr(means_out), _ptr(quats_out),
                                        _stream(stream)))
    return means_out, quats_out


def dgsm_crowd_frame(q_means, colors_in, colors_out, n_static, static_atlas, radii, rest_means, rest_quats,
                     scales, opac, quats_out, seg, poses, dyn_atlas, radii_dyn, lights, sh, centroids_out,
                     direct_frac=1.0, params=None, relight_params=None, timeout_barrier=-1,
                     ctx: Context | None = None, stream=None):
    """The moving-avatar frame as one persistent cooperative kernel
    (dgsm_crowd_frame): rigid motion, the dynamic atlases (tile 8, params
    max_pairs > 0), attenuation of every receiver by static x dynamic atlases,
    per-avatar centroids and relight.  q_means rows n_static.. receive the
    moved avatar means.  timeout_barrier 1..7 makes that grid barrier give up
    (DGSM_ERR_TIMEOUT in the status word)."""
    ctx = ctx or context(q_means.device.index)
    for t, nm, k in ((q_means, "q_means", 3), (colors_in, "colors_in", 3), (colors_out, "colors_out", 3),
                     (radii, "radii", None), (rest_means, "rest_means", 3), (rest_quats, "rest_quats", 4),
                     (scales, "scales", 3), (opac, "opac", None), (quats_out, "quats_out", 4),
                     (radii_dyn, "radii_dyn", None), (lights, "lights", 3), (sh, "sh", None),
                     (centroids_out, "centroids_out", 3)):
        _need(t, nm, shape_last=k)
    _need(static_atlas, "static_atlas")
    _need(dyn_atlas, "dyn_atlas")
    if poses.dtype != torch.float32 or not poses.is_contiguous() or tuple(poses.shape[1:]) != (8,):
        raise ValueError("poses must be a contiguous (n_obj, 8) float32 tensor")
    n_av = rest_means.shape[0]
    segs, n_obj = _segs(seg, n_av)
    L, K, H, W = static_atlas.shape
    Ld, Kd, Hd, Wd = dyn_atlas.shape
    if Ld != L or lights.shape[0] != L:
        raise ValueError("one static and one dynamic atlas per light")
    if q_means.shape[0] != n_static + n_av:
        raise ValueError("q_means holds the static receivers, then the avatars")
    a = CrowdFrameArgs()
    a.q_means, a.colors_in, a.colors_out, a.n_static = _ptr(q_means), _ptr(colors_in), _ptr(colors_out), n_static
    a.static_atlas, a.H, a.W, a.K, a.radii = _ptr(static_atlas), H, W, K, _ptr(radii)
    a.rest_means, a.rest_quats, a.scales, a.opac = _ptr(rest_means), _ptr(rest_quats), _ptr(scales), _ptr(opac)
    a.quats_out, a.n_avatar = _ptr(quats_out), n_av
    a.seg, a.n_obj, a.poses = C.cast(segs, C.c_void_p), n_obj, _ptr(poses)
    a.dyn_atlas, a.H_dyn, a.W_dyn, a.K_dyn, a.radii_dyn = _ptr(dyn_atlas), Hd, Wd, Kd, _ptr(radii_dyn)
    a.lights, a.L, a.sh, a.centroids_out = _ptr(lights), L, _ptr(sh), _ptr(centroids_out)
    a.direct_frac = float(direct_frac)
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    rp = relight_params if isinstance(relight_params, RelightParams) else RelightParams.make(**(relight_params or {}))
    ctx.check(_lib.dgsm_crowd_frame(ctx.handle, C.byref(a), C.byref(p), C.byref(rp), int(timeout_barrier),
                                    _stream(stream)))
    return colors_out


def dgsm_crowd_frame_phases(ctx: Context | None = None):
    """Milliseconds of the eight steps of the last profiled persistent frame
    (P1 prep .. P8 attenuation and relight)."""
    ctx = ctx or context()
    out = (C.c_double * 8)()
    ctx.check(_lib.dgsm_crowd_frame_phases(ctx.handle, out))
    return list(out)


class Graph:
    """A captured sequence of library calls (dgsm_graph); replay() relaunches it."""

    def __init__(self, ctx: Context, handle):
        self.ctx, self._h = ctx, handle

    def replay(self, stream):
        self.ctx.check(_lib.dgsm_graph_launch(self._h, _stream(stream)))

    def node_count(self) -> int:
        n = _i64(0)
        self.ctx.check(_lib.dgsm_graph_node_count(self._h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.dgsm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class capture:
    """with capture(stream, ctx) as cap: <library calls on stream>; then cap.graph.
    `stream` must be a torch.cuda.Stream other than the default stream."""

    def __init__(self, stream, ctx: Context | None = None):
        self.stream, self.ctx, self.graph = stream, ctx or context(), None

    def __enter__(self):
        self.ctx.check(_lib.dgsm_graph_begin(self.ctx.handle, _stream(self.stream)))
        return self

    def __exit__(self, et, ev, tb):
        h = _vp()
        rc = _lib.dgsm_graph_end(self.ctx.handle, _stream(self.stream), C.byref(h))
        if et is None:
            self.ctx.check(rc)
            self.graph = Graph(self.ctx, h)
        return False


def dgsm_autotune_build(means, scales, quats, opac, lights, H, W, radii, tiles=(8, 16),
                        chunks=(32, 64, 128, 192), reps=3, params=None, ctx: Context | None = None,
                        stream=None):
    """Measured tile x chunk choice for dgsm_build: (best Params, {(tile, chunk): ms})."""
    ctx = ctx or context(means.device.index)
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    L, K, n = lights.shape[0], radii.shape[0], means.shape[0]
    atlas = torch.empty((L, K, H, W), dtype=TORCH_DTYPES[p.atlas_dtype], device=means.device)
    ta = (C.c_int32 * len(tiles))(*tiles)
    ca = (C.c_int32 * len(chunks))(*chunks)
    ms = (C.c_float * (len(tiles) * len(chunks)))()
    best = Params()
    ctx.check(_lib.dgsm_autotune_build(ctx.handle, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac),
                                       n, _ptr(lights), L, H, W, _ptr(radii), K, C.byref(p), ta,
                                       len(tiles), ca, len(chunks), int(reps), _ptr(atlas),
                                       C.byref(best), ms, _stream(stream)))
    table = {(t, c): float(ms[a * len(chunks) + b]) for a, t in enumerate(tiles)
             for b, c in enumerate(chunks)}
    return best, table


def dgsm_selftest_wait(arrive: bool, limit: int = 4096, ctx: Context | None = None, stream=None):
    """One bounded mbarrier wait on the device (failure-detection self-test):
    without `arrive` it times out and records DGSM_ERR_TIMEOUT (read it with
    dgsm_sync_status)."""
    ctx = ctx or context()
    ctx.check(_lib.dgsm_selftest_wait(ctx.handle, 1 if arrive else 0, int(limit), _stream(stream)))


def dgsm_sync_status(ctx: Context | None = None, stream=None) -> int:
    ctx = ctx or context()
    rc = _lib.dgsm_sync_status(ctx.handle, _stream(stream))
    return rc


def dgsm_weighted_centroid(means, weights=None, ctx: Context | None = None, stream=None):
    """Alpha-weighted centroid (3,) float32 on the device."""
    ctx = ctx or context(means.device.index)
    _need(means, "means", shape_last=3)
    if weights is not None:
        _need(weights, "weights")
    out = torch.empty(3, dtype=torch.float32, device=means.device)
    ctx.check(_lib.dgsm_weighted_centroid(ctx.handle, _ptr(means), _ptr(weights), means.shape[0],
                                          _ptr(out), _stream(stream)))
    return out


def _host(t, name, dtype=torch.float32):
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} CPU tensor (pinned for async copies)")
    return t


def dgsm_frame_host(means, scales, quats, opac, colors, lights, H, W, radii, cube_dirs,
                    cube_rgb, cube_w, relight_range=(0, 0), lam=1e-3, params=None,
                    rparams=None, colors_out=None, sh_out=None, ctx: Context | None = None,
                    stream=None):
    """One frame from host tensors: shadowed + relit colours (host), SH (host)."""
    ctx = ctx or context()
    ts = dict(means=means, scales=scales, quats=quats, opac=opac, colors=colors, lights=lights,
              radii=radii, cube_dirs=cube_dirs, cube_rgb=cube_rgb, cube_w=cube_w)
    for k, t in ts.items():
        _host(t, k)
    n = means.shape[0]
    if colors_out is None:
        colors_out = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    if sh_out is None:
        sh_out = torch.empty((3, 9), dtype=torch.float32).pin_memory()
    fi = FrameHostIn(*(ts[k].data_ptr() for k in ("means", "scales", "quats", "opac", "colors")),
                     n, int(relight_range[0]), int(relight_range[1]), lights.data_ptr(),
                     lights.shape[0], H, W, radii.shape[0], radii.data_ptr(), cube_dirs.data_ptr(),
                     cube_rgb.data_ptr(), cube_w.data_ptr(), cube_dirs.shape[0], float(lam))
    p = params if isinstance(params, Params) else Params.make(**(params or {}))
    rp = rparams if isinstance(rparams, RelightParams) else RelightParams.make(**(rparams or {}))
    ctx.check(_lib.dgsm_frame_host(ctx.handle, C.byref(fi), C.byref(p), C.byref(rp),
                                   C.c_void_p(colors_out.data_ptr()), C.c_void_p(sh_out.data_ptr()),
                                   _stream(stream)))
    return colors_out, sh_out


class FrameQueue:
    """Pipelined host frames (dgsm_frame_host_submit / _wait) over two slots.

    submit(...) takes dgsm_frame_host's arguments and returns the slot; the
    host arrays and the outputs (pinned) must stay alive until wait(slot)."""

    def __init__(self, ctx: Context | None = None, stream=None):
        self.ctx, self.stream, self.next_slot = ctx or context(), stream, 0
        self._keep = [None, None]

    def submit(self, means, scales, quats, opac, colors, lights, H, W, radii, cube_dirs, cube_rgb, cube_w,
               relight_range=(0, 0), lam=1e-3, params=None, rparams=None, colors_out=None, sh_out=None):
        ts = dict(means=means, scales=scales, quats=quats, opac=opac, colors=colors, lights=lights,
                  radii=radii, cube_dirs=cube_dirs, cube_rgb=cube_rgb, cube_w=cube_w)
        for k, t in ts.items():
            _host(t, k)
        n = means.shape[0]
        if colors_out is None:
            colors_out = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        if sh_out is None:
            sh_out = torch.empty((3, 9), dtype=torch.float32).pin_memory()
        fi = FrameHostIn(*(ts[k].data_ptr() for k in ("means", "scales", "quats", "opac", "colors")),
                         n, int(relight_range[0]), int(relight_range[1]), lights.data_ptr(),
                         lights.shape[0], H, W, radii.shape[0], radii.data_ptr(), cube_dirs.data_ptr(),
                         cube_rgb.data_ptr(), cube_w.data_ptr(), cube_dirs.shape[0], float(lam))
        p = params if isinstance(params, Params) else Params.make(**(params or {}))
        rp = rparams if isinstance(rparams, RelightParams) else RelightParams.make(**(rparams or {}))
        slot = self.next_slot
        self.ctx.check(_lib.dgsm_frame_host_submit(self.ctx.handle, slot, C.byref(fi), C.byref(p), C.byref(rp),
                                                   C.c_void_p(colors_out.data_ptr()),
                                                   C.c_void_p(sh_out.data_ptr()), _stream(self.stream)))
        self._keep[slot] = (ts, colors_out, sh_out)
        self.next_slot = 1 - slot
        return slot

    def wait(self, slot):
        """The slot's (colors_out, sh_out) once its frame is complete."""
        self.ctx.check(_lib.dgsm_frame_host_wait(self.ctx.handle, slot))
        keep, self._keep[slot] = self._keep[slot], None
        return (keep[1], keep[2]) if keep else (None, None)


def dgsm_set_profiling(enable: bool, ctx: Context | None = None):
    ctx = ctx or context()
    ctx.check(_lib.dgsm_set_profiling(ctx.handle, int(bool(enable))))


def dgsm_measure_alu_peaks(ctx: Context | None = None, stream=None) -> dict:
    """Measured FP32 and MUFU lane-operation rates of the current GPU (blocks)."""
    ctx = ctx or context()
    out = (C.c_double * 4)()
    ctx.check(_lib.dgsm_measure_alu_peaks(ctx.handle, out, _stream(stream)))
    return {"fp32_ops_s": out[0], "ex2_ops_s": out[1], "rcp_ops_s": out[2], "rsqrt_ops_s": out[3]}


def dgsm_profile_collect(ctx: Context | None = None):
    """[(ms prep+binning+sort, ms tile kernel), ...] of the builds since the last call."""
    ctx = ctx or context()
    buf = (C.c_double * 512)()
    n = C.c_int(0)
    ctx.check(_lib.dgsm_profile_collect(ctx.handle, buf, 256, C.byref(n)))
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]


# ---- learned transmittance surrogate ---------------------------------------

def nf_param_count() -> int:
    return int(_lib.nf_param_count())


def nf_init(seed=0, n_lights=None, device=None, ctx: Context | None = None, stream=None):
    """Fresh parameters: (P,) or (n_lights, P) float32 on the device."""
    ctx = ctx or context(device)
    P = nf_param_count()
    shape = (P,) if n_lights is None else (n_lights, P)
    out = torch.empty(shape, dtype=torch.float32, device=torch.device("cuda", ctx.device))
    flat = out.view(-1, P)
    for l in range(flat.shape[0]):
        ctx.check(_lib.nf_init(ctx.handle, int(seed) + l, _ptr(flat[l]), _stream(stream)))
    return out


def nf_loss_grad(params, uvr, target, ctx: Context | None = None, stream=None):
    """(loss (1,), grad (P,)) of the field's MSE at explicit inputs."""
    ctx = ctx or context(params.device.index)
    _need(params, "params")
    _need(uvr, "uvr", shape_last=3)
    _need(target, "target")
    loss = torch.zeros(1, dtype=torch.float32, device=params.device)
    grad = torch.empty_like(params)
    ctx.check(_lib.nf_loss_grad(ctx.handle, _ptr(params), _ptr(uvr), _ptr(target), uvr.shape[0],
                                _ptr(loss), _ptr(grad), _stream(stream)))
    return loss, grad


def nf_train(atlas_l, params, adam_m, adam_v, steps, batch=8192, lr=1e-3, seed=0, step0=0,
             ctx: Context | None = None, stream=None):
    """Adam steps on one light's atlas [K][H][W]; returns the per-step losses."""
    ctx = ctx or context(params.device.index)
    _need(atlas_l, "atlas_l")
    K, H, W = atlas_l.shape
    loss = torch.zeros(max(steps, 1), dtype=torch.float32, device=params.device)
    ctx.check(_lib.nf_train(ctx.handle, _ptr(atlas_l), H, W, K, _ptr(params), _ptr(adam_m),
                            _ptr(adam_v), int(steps), int(batch), float(lr), int(seed), int(step0),
                            _ptr(loss), _stream(stream)))
    return loss[:steps]


def nf_forward(params, uvr, ctx: Context | None = None, stream=None):
    ctx = ctx or context(params.device.index)
    _need(params, "params")
    _need(uvr, "uvr", shape_last=3)
    out = torch.empty(uvr.shape[0], dtype=torch.float32, device=uvr.device)
    ctx.check(_lib.nf_forward(ctx.handle, _ptr(params), _ptr(uvr), uvr.shape[0], _ptr(out),
                              _stream(stream)))
    return out


def nf_tile_error(params, atlas_l, tile=8, ctx: Context | None = None, stream=None):
    ctx = ctx or context(params.device.index)
    K, H, W = atlas_l.shape
    out = torch.empty(((H + tile - 1) // tile) * ((W + tile - 1) // tile), dtype=torch.float32,
                      device=atlas_l.device)
    ctx.check(_lib.nf_tile_error(ctx.handle, _ptr(params), _ptr(atlas_l), H, W, K, tile, _ptr(out),
                                 _stream(stream)))
    return out


def nf_attenuate(params, radii, lights, q_means, colors, H, W, mask=None, atlas=None, tile=8,
                 light_w=None, direct_frac=1.0, out=None, want_T=False, ctx: Context | None = None,
                 stream=None):
    """Attenuation through the per-light fields params (L, P); see dgsm_attenuate."""
    ctx = ctx or context(params.device.index)
    _need(params, "params")
    L = lights.shape[0]
    Q = q_means.shape[0]
    if out is None:
        out = torch.empty_like(colors)
    T = torch.empty((Q, L), dtype=torch.float32, device=colors.device) if want_T else None
    ctx.check(_lib.nf_attenuate(ctx.handle, _ptr(params), _ptr(mask), _ptr(atlas), L, H, W,
                                _ptr(radii), radii.shape[0], tile, _ptr(lights), _ptr(q_means),
                                _ptr(colors), Q, _ptr(light_w), float(direct_frac), _ptr(out),
                                _ptr(T), _stream(stream)))
    return (out, T) if want_T else out
