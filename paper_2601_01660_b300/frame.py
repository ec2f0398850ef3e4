"""Per-frame pipeline of the moving-avatar workload, as library calls.

A static scene (its atlases built once) is shadowed together with moving
avatars whose atlases are rebuilt every frame:

  1. rigid motion of every avatar to this frame's pose (dgsm_rigid_transform);
  2. the avatars' dynamic atlases for all lights in one build
     (dgsm_build with max_pairs, so that nothing waits on the host);
  3. per-avatar alpha-weighted centroids and the SH relight of the avatars
     (dgsm_segment_centroids, sh_relight_objects; Sec. 3.5), on a side
     stream beside step 2, which they do not need;
  4. attenuation of every Gaussian, static and avatar (relit), by
     T_static * T_dynamic (dgsm_attenuate_dyn; Sec. 3.3).

The relight and the attenuation each scale a Gaussian's colour by a
non-negative factor (Eq. 10's max(0, gamma c s); 1 - w_d + w_d sum_l w_l T_l),
so relighting first gives the same colours as relighting the attenuated ones.

With persistent=True the four steps run as ONE persistent cooperative
kernel (dgsm_crowd_frame: grid-wide barriers between the steps instead of
kernel boundaries, tile 8, capacity build).

`capture()` records these calls once into CUDA graphs; a frame is then one
graph launch.  Two graphs alternate between two pinned pose buffers, so the
host writes the poses of frame f + 1 while frame f runs.  Every step runs in
the library's kernels; this module only owns buffers and orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native


def _dev(a, device):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device)


class CrowdFrame:
    def __init__(self, static, avatars, seg, lights, H, W, radii, H_dyn, W_dyn, radii_dyn, sh,
                 build_params=None, relight_params=None, device="cuda", ctx=None, persistent=False):
        self.nat = nat = native()
        self.persistent = persistent
        self.timeout_barrier = -1  # 1..7: that grid barrier of the persistent kernel gives up
        self.device = torch.device(device)
        self.ctx = ctx or nat.Context(self.device.index or 0)
        self.stream = torch.cuda.Stream(device=self.device)
        self.side = torch.cuda.Stream(device=self.device)  # the relight, beside the dynamic build
        self.seg = [int(x) for x in seg]
        self.n_static, self.n_dyn = static.n, avatars.n
        self.H, self.W, self.H_dyn, self.W_dyn = H, W, H_dyn, W_dyn
        self.bp = dict(build_params or {})
        self.rp = dict(relight_params or {})
        dv = self.device
        n = self.n_static + self.n_dyn
        # receivers: static Gaussians first, then the avatars (rewritten per frame)
        self.q_means = torch.empty((n, 3), dtype=torch.float32, device=dv)
        self.q_means[: self.n_static] = _dev(static.means, dv)
        self.colors_in = _dev(np.concatenate([static.colors, avatars.colors]), dv)
        self.colors_mid = self.colors_in.clone()  # the attenuation's input: avatar rows relit per frame
        self.colors_out = torch.empty_like(self.colors_in)
        self.av_means = self.q_means[self.n_static:]
        self.rest_means = _dev(avatars.means, dv)
        self.rest_quats = _dev(avatars.quats, dv)
        self.av_quats = torch.empty_like(self.rest_quats)
        self.av_scales = _dev(avatars.scales, dv)
        self.av_opac = _dev(avatars.opac, dv)
        self.lights = _dev(lights, dv)
        self.radii = _dev(radii, dv)
        self.radii_dyn = _dev(radii_dyn, dv)
        self.sh = sh if torch.is_tensor(sh) else _dev(np.float32(sh), dv)
        self.centroids = torch.empty((len(self.seg) - 1, 3), dtype=torch.float32, device=dv)
        L = self.lights.shape[0]
        self.dyn_atlas = torch.empty((L, self.radii_dyn.shape[0], H_dyn, W_dyn), dtype=torch.float32,
                                     device=dv)
        self.poses = [torch.zeros((len(self.seg) - 1, 8), dtype=torch.float32).pin_memory()
                      for _ in range(2)]
        self.done = [None, None]
        self.graphs = None
        self.frame = 0
        # the static atlases, built once from the static occluders
        self.stream.wait_stream(torch.cuda.current_stream(dv))
        with torch.cuda.stream(self.stream):
            sd = {k: _dev(getattr(static, k), dv) for k in ("scales", "quats", "opac")}
            self.static_atlas = nat.dgsm_build(self.q_means[: self.n_static], sd["scales"], sd["quats"],
                                               sd["opac"], self.lights, H, W, self.radii,
                                               params=dict(self.bp, max_pairs=0), ctx=self.ctx,
                                               stream=self.stream)
        self.stream.synchronize()

    # -- one frame as library calls ------------------------------------------
    def _calls(self, poses, max_pairs):
        nat, s, ctx = self.nat, self.stream, self.ctx
        if self.persistent and max_pairs > 0:
            nat.dgsm_crowd_frame(self.q_means, self.colors_in, self.colors_out, self.n_static, self.static_atlas,
                                 self.radii, self.rest_means, self.rest_quats, self.av_scales, self.av_opac,
                                 self.av_quats, self.seg, poses, self.dyn_atlas, self.radii_dyn, self.lights,
                                 self.sh, self.centroids, params=dict(self.bp, tile=8, max_pairs=max_pairs),
                                 relight_params=self.rp, timeout_barrier=self.timeout_barrier, ctx=ctx, stream=s)
            return
        nat.dgsm_rigid_transform(self.rest_means, self.rest_quats, self.seg, poses,
                                 means_out=self.av_means, quats_out=self.av_quats, ctx=ctx, stream=s)
        side = self.side
        side.wait_stream(s)  # the moved avatars
        nat.dgsm_segment_centroids(self.av_means, self.av_opac, self.seg, out=self.centroids, ctx=ctx,
                                   stream=side)
        av_mid = self.colors_mid[self.n_static:]
        nat.sh_relight_objects(self.sh, self.av_means, self.av_quats, self.av_scales,
                               self.colors_in[self.n_static:], self.centroids, self.seg, params=self.rp,
                               out=av_mid, ctx=ctx, stream=side)
        nat.dgsm_build(self.av_means, self.av_scales, self.av_quats, self.av_opac, self.lights,
                       self.H_dyn, self.W_dyn, self.radii_dyn, params=dict(self.bp, max_pairs=max_pairs),
                       out=self.dyn_atlas, ctx=ctx, stream=s)
        s.wait_stream(side)
        nat.dgsm_attenuate_dyn(self.static_atlas, self.radii, self.dyn_atlas, self.radii_dyn, self.lights,
                               self.q_means, self.colors_mid, out=self.colors_out, ctx=ctx, stream=s)

    def _write_poses(self, poses):
        """This frame's pinned pose buffer, filled once the frame that last
        read it has run."""
        k = self.frame & 1
        if self.done[k] is not None:
            self.done[k].synchronize()
        self.poses[k].copy_(torch.as_tensor(poses))
        return k

    def _frame_done(self, k):
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self.done[k] = ev
        self.frame += 1

    def size_pairs(self, pose_list, headroom=1.25):
        """Pair capacity of the dynamic build: the largest exact pair count
        (tile and super-tile pairs) over the given poses, with headroom."""
        best = 0
        for p in pose_list:
            self.step_eager(p)
            self.stream.synchronize()
            st = self.nat.dgsm_get_build_stats(self.ctx)
            best = max(best, st["n_pairs"], st["n_super_pairs"])
        self.max_pairs = int(best * headroom) + 1024
        return self.max_pairs

    def autotune(self, poses, tiles=(8, 16), chunks=(32, 64, 128), reps=3):
        """Measured tile x chunk of the dynamic build at `poses`; keeps the best."""
        k = self._write_poses(poses)
        nat = self.nat
        nat.dgsm_rigid_transform(self.rest_means, self.rest_quats, self.seg, self.poses[k],
                                 means_out=self.av_means, quats_out=self.av_quats, ctx=self.ctx,
                                 stream=self.stream)
        best, table = nat.dgsm_autotune_build(self.av_means, self.av_scales, self.av_quats, self.av_opac,
                                              self.lights, self.H_dyn, self.W_dyn, self.radii_dyn,
                                              tiles=tiles, chunks=chunks, reps=reps, params=self.bp,
                                              ctx=self.ctx, stream=self.stream)
        self._frame_done(k)
        self.bp.update(tile=best.tile, chunk=best.chunk)
        return (best.tile, best.chunk), table

    def step_eager(self, poses, max_pairs=None):
        """One frame by direct calls (max_pairs None: the exact, blocking build)."""
        k = self._write_poses(poses)
        self._calls(self.poses[k], 0 if max_pairs is None else max_pairs)
        self._frame_done(k)

    def capture(self):
        """Record the frame into two graphs (one per pinned pose buffer)."""
        if not hasattr(self, "max_pairs"):
            raise RuntimeError("size_pairs() first")
        # run once uncaptured so that the workspace reaches its size
        self._calls(self.poses[0], self.max_pairs)
        self.stream.synchronize()
        self.done = [None, None]
        self.graphs = []
        for k in range(2):
            with self.nat.capture(self.stream, self.ctx) as cap:
                self._calls(self.poses[k], self.max_pairs)
            self.graphs.append(cap.graph)
        self.frame = 0
        return sum(g.node_count() for g in self.graphs) // 2

    def step_graph(self, poses):
        """Write this frame's poses and launch its graph (asynchronous)."""
        k = self._write_poses(poses)
        self.graphs[k].replay(self.stream)
        self._frame_done(k)

    def close(self):
        if self.graphs:
            for g in self.graphs:
                g.close()
            self.graphs = None
