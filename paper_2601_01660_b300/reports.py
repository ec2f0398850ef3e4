"""Reports beside the benchmark step (each prints one JSON line via bench.py).

  precision  3M-Gaussian cube scene, 4 lights, 64x64x16 atlases stored as
             float32 / float16 / bfloat16 (tau always accumulated in float32):
             per-light max and mean |dT| of the 16-bit stores against float32
             over every voxel, build times.
  surrogate  the learned transmittance field trained on 512x512x64 atlases of
             the 20k-Gaussian cube scene with 4 lights, then used to attenuate
             3M Gaussians: |dT| p50/p99 against the exact atlas lookup, with
             and without the per-tile exact fallback, memory footprint,
             Gaussians/s, and an atlas of the same memory as the weights.
  field      the surrogate's tensor-core forward pass alone: 3M inputs
             (u, v, rho) through one light's field (GPU-initialised weights),
             TFLOP/s against the measured bf16 peak.
  frame      the moving-avatar workload (1.5M static Gaussians with 4-light
             512x512x64 atlases built once, 8 avatars of 100k walking for
             120 frames, 256x256x32 dynamic atlases per frame, 2.3M
             attenuated, 800k relit): autotuned tile x chunk of the dynamic
             build, then ms per frame for direct calls with the blocking
             build, direct calls with the capacity build, and graph replay,
             with a per-stage breakdown.

Comparisons against the FP64 oracle live in the test suite.
"""
from __future__ import annotations

import json
import time

import numpy as np


def _dev(a, torch):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _time(torch, fn, reps=5):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def precision() -> dict:
    """Storage precision on the GPU: float16 / bfloat16 atlases against the
    float32 atlas over every voxel (the float32 atlas itself is checked
    against the FP64 oracle by the test suite)."""
    import torch

    from paper_2601_01660_b300 import native, scenes
    nat = native()
    wl = scenes.workload("cube3m4l")
    sc, lights, radii, H, W = wl["occluders"], wl["lights"], wl["radii"], wl["H"], wl["W"]
    d = {k: _dev(getattr(sc, k), torch) for k in ("means", "scales", "quats", "opac")}
    lt, rt = _dev(lights, torch), _dev(radii, torch)
    atl, times = {}, {}
    for dt in ("f32", "f16", "bf16"):
        f = lambda: nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lt, H, W, rt,
                                   params=dict(atlas_dtype=dt))
        atl[dt] = f()
        times[dt] = _time(torch, f, reps=3)
    L = lights.shape[0]
    out = {"report": "precision", "workload": "cube3m4l: 3M Gaussians, 4 lights, 64x64x16",
           "build_ms": {k: round(v, 3) for k, v in times.items()}, "abs_dT_vs_f32": {}}
    ref = atl["f32"].double()
    for dt in ("f16", "bf16"):
        err = (atl[dt].double() - ref).abs()
        out["abs_dT_vs_f32"][dt] = {f"light{l}": {"max": float(err[l].max()), "mean": float(err[l].mean())}
                                    for l in range(L)}
    return out


# Adam steps and learning rate of the field's training, in phases (a decaying
# rate: the last phases settle the fit near shadow edges)
SURROGATE_SCHEDULE = ((6000, 2e-3), (3000, 5e-4), (1000, 1e-4))


def _small_tile_error(nat, torch, small, small_r, light, atlas_l, radii, H, W, tile):
    """Largest |T_small - T| over each tile's voxels of a light's exact atlas,
    T_small the trilinear lookup of a coarse atlas at every voxel centre."""
    j = (2 * torch.arange(W, device="cuda", dtype=torch.float64) + 1) / W - 1
    i = (2 * torch.arange(H, device="cuda", dtype=torch.float64) + 1) / H - 1
    v, u = torch.meshgrid(i, j, indexing="ij")
    z = 1 - u.abs() - v.abs()
    x = torch.where(z < 0, torch.where(u >= 0, 1.0, -1.0) * (1 - v.abs()), u)
    y = torch.where(z < 0, torch.where(v >= 0, 1.0, -1.0) * (1 - u.abs()), v)
    dirs = torch.stack([x, y, z], -1)
    dirs = (dirs / dirs.norm(dim=-1, keepdim=True)).float()
    err = torch.zeros(H // tile, W // tile, device="cuda")
    for k in range(radii.shape[0]):
        pts = (light[None, None, :] + radii[k] * dirs).reshape(-1, 3).contiguous()
        _, T = nat.dgsm_attenuate(small, small_r, light[None].contiguous(), pts, torch.ones_like(pts),
                                  want_T=True)
        e = (T[:, 0].reshape(H, W) - atlas_l[k]).abs()
        err = torch.maximum(err, e.reshape(H // tile, tile, W // tile, tile).amax(dim=(1, 3)))
    return err.flatten()


def surrogate(schedule=SURROGATE_SCHEDULE, batch: int = 16384, n_query: int = 3_000_000,
              tol: float = 0.02) -> dict:
    import torch

    from paper_2601_01660_b300 import native, scenes
    nat = native()
    occ = scenes.cube_scene(20_000, seed=0)
    lights = scenes.four_lights()
    H = W = 512
    K = 64
    radii = scenes.radii_geometric(0.05, 12.0, K)
    d = {k: _dev(getattr(occ, k), torch) for k in ("means", "scales", "quats", "opac")}
    lt, rt = _dev(lights, torch), _dev(radii, torch)
    atlas = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lt, H, W, rt)
    L = lights.shape[0]
    P = nat.nf_param_count()
    params = nat.nf_init(seed=100, n_lights=L)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for l in range(L):
        m, v = torch.zeros(P, device="cuda"), torch.zeros(P, device="cuda")
        step0, ls = 0, []
        for steps, lr in schedule:
            ls.append(nat.nf_train(atlas[l], params[l], m, v, steps=steps, batch=batch, lr=lr,
                                   seed=l + 1, step0=step0).cpu().numpy())
            step0 += steps
        losses.append(np.concatenate(ls))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    tile = 8
    n_tiles = (H // tile) * (W // tile)
    errs = torch.stack([nat.nf_tile_error(params[l], atlas[l], tile=tile) for l in range(L)])
    mask = (errs > tol).to(torch.uint8).contiguous()
    q = scenes.cube_scene(n_query, seed=7)
    qm, qc = _dev(q.means, torch), _dev(q.colors, torch)
    _, T_ex = nat.dgsm_attenuate(atlas, rt, lt, qm, qc, want_T=True)
    _, T_nf = nat.nf_attenuate(params, rt, lt, qm, qc, H, W, want_T=True)
    _, T_fb = nat.nf_attenuate(params, rt, lt, qm, qc, H, W, mask=mask, atlas=atlas, want_T=True)
    # an exact atlas with the weights' memory: bfloat16 weights, float32 voxels
    weight_bytes = L * (P - 1) * 2 + L * 4
    side = int(np.sqrt(weight_bytes / (L * 4 * 16)))
    small_r = _dev(scenes.radii_geometric(0.05, 12.0, 16), torch)
    small = nat.dgsm_build(d["means"], d["scales"], d["quats"], d["opac"], lt, side, side, small_r)
    _, T_sm = nat.dgsm_attenuate(small, small_r, lt, qm, qc, want_T=True)
    # the same fallback rule on the equal-memory atlas
    errs_sm = torch.stack([_small_tile_error(nat, torch, small[l:l + 1].contiguous(), small_r, lt[l], atlas[l],
                                             rt, H, W, tile) for l in range(L)])
    fb_small = float((errs_sm > tol).float().mean().item())

    def stats(T):
        e = (T - T_ex).abs().flatten().cpu().numpy()
        return {"p50": float(np.quantile(e, 0.5)), "p99": float(np.quantile(e, 0.99)),
                "max": float(e.max())}

    t_ex = _time(torch, lambda: nat.dgsm_attenuate(atlas, rt, lt, qm, qc))
    t_nf = _time(torch, lambda: nat.nf_attenuate(params, rt, lt, qm, qc, H, W))
    t_fb = _time(torch, lambda: nat.nf_attenuate(params, rt, lt, qm, qc, H, W, mask=mask, atlas=atlas))
    fb_frac = float(mask.float().mean().item())
    atlas_bytes = atlas.numel() * 4
    return {
        "report": "surrogate",
        "workload": f"cube20k occluders, 4 lights, exact atlases 4x{H}x{W}x{K}; {n_query} queries",
        "training": {"schedule_steps_lr": [list(x) for x in schedule], "batch": batch,
                     "seconds_total": round(t_train, 2),
                     "loss_first": [float(x[:10].mean()) for x in losses],
                     "loss_last": [float(x[-50:].mean()) for x in losses]},
        "abs_dT_vs_exact": {"field": stats(T_nf), f"field+fallback(tol {tol})": stats(T_fb),
                            f"exact atlas {side}x{side}x16 (same bytes as the weights)": stats(T_sm)},
        "fallback_tile_fraction": {"field": fb_frac, "equal_memory_atlas": fb_small,
                                   "rule": f"a tile keeps its exact voxels when its largest error exceeds {tol}"},
        "memory_bytes": {"exact_atlases": atlas_bytes, "field_weights_bf16": weight_bytes,
                         "field+fallback_tiles": weight_bytes + int(fb_frac * atlas_bytes),
                         "equal_memory_atlas": int(small.numel() * 4),
                         "equal_memory_atlas+fallback_tiles": int(small.numel() * 4) + int(fb_small * atlas_bytes)},
        "gaussians_per_s": {"exact": n_query / (t_ex * 1e-3), "field": n_query / (t_nf * 1e-3),
                            "field+fallback": n_query / (t_fb * 1e-3)},
        "ms": {"exact": t_ex, "field": t_nf, "field+fallback": t_fb},
    }


def frame(frames: int = 120, workload: str = "crowd8") -> dict:
    import torch

    from paper_2601_01660_b300 import layout, native, scenes
    from paper_2601_01660_b300.frame import CrowdFrame
    nat = native()
    wl = scenes.workload(workload)
    # storage order: the room and each avatar in the Z-order of their means
    wl["static"], _ = layout.zorder_scene(nat, wl["static"], [0, wl["static"].n], "cuda")
    wl["avatars"], _ = layout.zorder_scene(nat, wl["avatars"], [int(x) for x in wl["seg"]], "cuda")
    D, Y, w = wl["cubemap"]
    sh = nat.sh_fit(_dev(D, torch), _dev(Y, torch), _dev(w, torch))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cf = CrowdFrame(wl["static"], wl["avatars"], wl["seg"], wl["lights"], wl["H"], wl["W"], wl["radii"],
                    wl["H_dyn"], wl["W_dyn"], wl["radii_dyn"], sh)
    t_static = time.perf_counter() - t0
    mo = wl["motion"]
    poses = [scenes.avatar_poses(mo, f) for f in range(frames)]
    (tile, chunk), table = cf.autotune(poses[0])
    cf.size_pairs(poses[::10])
    s = cf.stream

    def run(step, n):
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = time.perf_counter()
        e0.record(s)
        for f in range(n):
            step(poses[f % frames])
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / n, (time.perf_counter() - t) * 1e3 / n

    for _ in range(3):
        cf.step_eager(poses[0])
    ms_sync, wall_sync = run(lambda p: cf.step_eager(p), frames)
    ms_cap, wall_cap = run(lambda p: cf.step_eager(p, max_pairs=cf.max_pairs), frames)
    nodes = cf.capture()
    for _ in range(3):
        cf.step_graph(poses[0])
    ms_graph, wall_graph = run(cf.step_graph, frames)
    status = nat.dgsm_sync_status(cf.ctx, stream=s)
    # per-stage times of one frame (capacity build, direct calls), one stage
    # after the other on one stream (a frame runs the centroids and the relight
    # beside the dynamic build)
    k = cf._write_poses(poses[7])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record(s)
    nat.dgsm_rigid_transform(cf.rest_means, cf.rest_quats, cf.seg, cf.poses[k], means_out=cf.av_means,
                             quats_out=cf.av_quats, ctx=cf.ctx, stream=s)
    ev[1].record(s)
    nat.dgsm_build(cf.av_means, cf.av_scales, cf.av_quats, cf.av_opac, cf.lights, cf.H_dyn, cf.W_dyn,
                   cf.radii_dyn, params=dict(cf.bp, max_pairs=cf.max_pairs), out=cf.dyn_atlas, ctx=cf.ctx,
                   stream=s)
    ev[2].record(s)
    nat.dgsm_segment_centroids(cf.av_means, cf.av_opac, cf.seg, out=cf.centroids, ctx=cf.ctx, stream=s)
    ev[3].record(s)
    av_mid = cf.colors_mid[cf.n_static:]
    nat.sh_relight_objects(cf.sh, cf.av_means, cf.av_quats, cf.av_scales, cf.colors_in[cf.n_static:],
                           cf.centroids, cf.seg, out=av_mid, ctx=cf.ctx, stream=s)
    ev[4].record(s)
    nat.dgsm_attenuate_dyn(cf.static_atlas, cf.radii, cf.dyn_atlas, cf.radii_dyn, cf.lights, cf.q_means,
                           cf.colors_mid, out=cf.colors_out, ctx=cf.ctx, stream=s)
    ev[5].record(s)
    cf._frame_done(k)
    ev[5].synchronize()
    stats = nat.dgsm_get_build_stats(cf.ctx)
    names = ["rigid_transform", "dynamic_build", "centroids", "relight", "attenuate_static_x_dynamic"]
    stages = {nm: ev[i].elapsed_time(ev[i + 1]) for i, nm in enumerate(names)}
    cf.close()
    # the same frames as one persistent cooperative kernel (tile 8), direct and in a graph
    cf.persistent = True
    if cf.bp.get("tile", 8) != 8:  # the persistent kernel bins with tile 8: capacity for that
        cf.bp.update(tile=8)
        cf.size_pairs(poses[::10])
    for _ in range(3):
        cf.step_eager(poses[0], max_pairs=cf.max_pairs)
    ms_pk, wall_pk = run(lambda p: cf.step_eager(p, max_pairs=cf.max_pairs), frames)
    status_pk = nat.dgsm_sync_status(cf.ctx, stream=s)
    nodes_pk = cf.capture()
    for _ in range(3):
        cf.step_graph(poses[0])
    ms_pkg, wall_pkg = run(cf.step_graph, frames)
    status_pkg = nat.dgsm_sync_status(cf.ctx, stream=s)
    cf.close()
    # its eight steps (global-timer stamps at the grid barriers), median of 5 frames
    nat.dgsm_set_profiling(True, ctx=cf.ctx)
    ph = []
    for f in range(5):
        cf.step_eager(poses[7 + f], max_pairs=cf.max_pairs)
        ph.append(nat.dgsm_crowd_frame_phases(cf.ctx))
    nat.dgsm_set_profiling(False, ctx=cf.ctx)
    ph = [sorted(x[k] for x in ph)[2] for k in range(8)]
    phase_names = ["P1_motion_prep_super_counts", "P2_key_offsets_units_centroids", "P3_super_lists",
                   "P4_fine_binning", "P5_tile_offsets_items", "P6_tile_lists", "P7_tiles_closed_form",
                   "P8_attenuate_relight"]
    return {
        "report": "frame",
        "workload": (f"{workload}: {wl['static'].n} static + 8 x {wl['avatars'].n // 8} avatar Gaussians, 4 lights; "
                     "static 512x512x64 (built once), dynamic 256x256x32 per frame; all attenuated, the avatars "
                     "relit"),
        "frames": frames, "static_build_s": round(t_static, 3),
        "autotune_ms": {f"tile{t}_chunk{c}": round(v, 3) for (t, c), v in table.items()},
        "chosen": {"tile": tile, "chunk": chunk}, "max_pairs": cf.max_pairs,
        "dynamic_build_pairs": stats["n_pairs"], "dynamic_ray_evals": stats["ray_evals"],
        "ms_per_frame": {"direct_blocking_build": round(ms_sync, 3), "direct_capacity_build": round(ms_cap, 3),
                         "graph_replay": round(ms_graph, 3), "persistent_kernel": round(ms_pk, 3),
                         "persistent_kernel_graph": round(ms_pkg, 3)},
        "host_ms_per_frame": {"direct_blocking_build": round(wall_sync, 3),
                              "direct_capacity_build": round(wall_cap, 3), "graph_replay": round(wall_graph, 3),
                              "persistent_kernel": round(wall_pk, 3), "persistent_kernel_graph": round(wall_pkg, 3)},
        "graph_nodes_per_frame": nodes, "status_after_replay": status,
        "persistent_graph_nodes_per_frame": nodes_pk, "persistent_status": [status_pk, status_pkg],
        "persistent_phase_ms": {nm: round(v, 4) for nm, v in zip(phase_names, ph)},
        "stage_ms": {k2: round(v, 4) for k2, v in stages.items()},
    }


def field(n: int = 3_000_000, reps: int = 20) -> dict:
    import os

    import torch

    from paper_2601_01660_b300 import native
    nat = native()
    params = nat.nf_init(seed=5, n_lights=1)[0].contiguous()
    g = torch.Generator(device="cuda").manual_seed(9)
    uvr = torch.rand(n, 3, device="cuda", generator=g)
    uvr[:, :2] = uvr[:, :2] * 2 - 1
    ms = _time(torch, lambda: nat.nf_forward(params, uvr), reps=reps)
    flop = n * 2.0 * (96 * 64 + 3 * 64 * 64 + 64)
    peak = None
    try:
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        peak = float(json.load(open(os.path.join(root, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        pass
    tf = flop / (ms * 1e-3) / 1e12
    return {"report": "field", "inputs": n, "ms": round(ms, 4), "field_evals_per_s": n / (ms * 1e-3),
            "tflops": round(tf, 2), "bf16_peak_tflops": peak,
            "frac": round(tf / peak, 4) if peak else None,
            "flop_per_eval": 2 * (96 * 64 + 3 * 64 * 64 + 64), "kernel": "tc::field_kernel<MODE_UVR> (tcgen05)"}


def main(which: str, frame_workload: str = "crowd8") -> None:
    if which == "frame":
        print(json.dumps(frame(workload=frame_workload)), flush=True)
        return
    fn = {"precision": precision, "surrogate": surrogate, "field": field}[which]
    print(json.dumps(fn()), flush=True)
