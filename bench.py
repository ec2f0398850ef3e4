#!/usr/bin/env python3
"""Benchmark of the Deep Gaussian Shadow Map hot path on B300.

One step = one pass of every hot-path row over the indoor-room workload
(1.5M room Gaussians + a 100k-Gaussian avatar, one light at 2.8 m):
DGSM build of a 512x512x64 atlas (prep, light-space tile binning, radix sort,
closed-form tile kernel), attenuation of all 1.6M Gaussians, FP64 SH probe fit
on 6x64^2 cubemap samples, and the radiance transfer of the avatar.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  metric = Gaussian-ray evaluations per second over the
whole step (an evaluation is one texel ray x one Gaussian whose culling
ellipsoid that ray cuts at t > 0, i.e. the pairs the method must evaluate);
the line also carries ms per 512^2x64 build and attenuated Gaussians/s.
Under torchrun each rank runs its own light (independent problems: weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gaussian-ray evals/s and ms per 512²×64 DGSM build; attenuated Gaussians/s"
UNIT = "Gaussian-ray evals/s"
WORKLOAD = "room1p6m"

# Algorithmic single-precision work of the build tile kernel, per unit, as
# the measurement plan fixes it (arithmetic a minimal implementation of the
# closed form must issue):
#   per Gaussian-ray evaluation: 45-55 FP32 (whitened direction 18, a and b 12,
#     cross product and norm 14, the rest), counted as 50, + 1 rsqrt + 1 ex2
#   per shell evaluation (Eq. 3 at one radius): 20 FP32 + 1 rcp + 1 ex2
#   per voxel: 1 FP32 (prefix sum) + 1 ex2
# MUFU instructions differ in rate (ex2 runs at twice the rate of rcp and
# rsqrt on this part), so the MUFU roofline weighs each by its measured rate.
FP32_PER_EVAL, RSQ_PER_EVAL, EX2_PER_EVAL = 50, 1, 1
FP32_PER_SHELL, RCP_PER_SHELL, EX2_PER_SHELL = 20, 1, 1
FP32_PER_VOXEL, EX2_PER_VOXEL = 1, 1
TILE_KERNEL = "build_tiles_kernel"
L2_BYTES = 126 * 1024 * 1024


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def load_workload(rank: int, name: str = WORKLOAD):
    from paper_2601_01660_b300 import scenes, shard
    wl = scenes.workload(name)
    wl["lights"] = shard.offset_light(wl["lights"], rank)  # each rank: its own light
    return wl


def step_config(wl, workload, world):
    """The workload's description in the JSON line (both arms)."""
    sc = wl["occluders"]
    av = sc.meta["avatar"]
    H, W, K = wl["H"], wl["W"], wl["radii"].shape[0]
    return {"workload": workload, "gaussians": int(sc.n), "avatar_gaussians": int(av.stop - av.start),
            "lights_per_rank": int(wl["lights"].shape[0]), "atlas": [H, W, K], "shells": "geometric 0.05-12 m",
            "cubemap_samples": int(wl["cubemap"][0].shape[0]), "relight_grid": [32, 64],
            "l2": "flushed between steps (2x L2 write), outside the timed events",
            "parallelism": f"{world} independent light(s), one per GPU"}


# ----------------------------------------------------------------------------- ours

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2601_01660_b300 import native
    nat = native()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = load_workload(rank, args.workload)
    # storage order: the Z-order of the means within the room and within the
    # avatar, taken once at load (outside every timed region); the scene as
    # generated is kept to time the attenuation in its order too
    from paper_2601_01660_b300 import layout
    sc0 = wl["occluders"]
    wl["occluders"], _ = layout.zorder_scene(nat, sc0, layout.room_parts(sc0), dev)
    sc = wl["occluders"]
    av_slice = sc.meta["avatar"]
    a0, a1 = av_slice.start, av_slice.stop
    H, W, radii_np, lights_np = wl["H"], wl["W"], wl["radii"], wl["lights"]
    K, L, N = radii_np.shape[0], lights_np.shape[0], sc.n
    D_np, Y_np, w_np = wl["cubemap"]
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    means, scales, quats, opac, colors = (t(getattr(sc, k)) for k in
                                          ("means", "scales", "quats", "opac", "colors"))
    lights, radii = t(lights_np), t(radii_np)
    D, Y, w = t(D_np), t(Y_np), t(w_np)
    atlas = torch.empty((L, K, H, W), dtype=torch.float32, device=dev)
    out = torch.empty_like(colors)
    sh = None
    stream = torch.cuda.current_stream()
    ev_att = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    att_ms = []

    def step(time_att=False):
        nat.dgsm_build(means, scales, quats, opac, lights, H, W, radii, out=atlas)
        if time_att:
            ev_att[0].record(stream)
        nat.dgsm_attenuate(atlas, radii, lights, means, colors, out=out)
        if time_att:
            ev_att[1].record(stream)
        s = nat.sh_fit(D, Y, w)
        cen = nat.dgsm_weighted_centroid(means[a0:a1], opac[a0:a1])
        nat.sh_relight(s, means[a0:a1], quats[a0:a1], scales[a0:a1], out[a0:a1], cen,
                       out=out[a0:a1])
        return s

    for _ in range(args.warmup):
        sh = step()
    torch.cuda.synchronize()
    stats = nat.dgsm_get_build_stats()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]
    # roofline denominators of the tile kernel: FP32 and MUFU rates measured
    # now, on this GPU, with the SM clock sampled meanwhile
    with ClockSampler(gpu_index) as pclk:
        peaks = nat.dgsm_measure_alu_peaks()
    peaks["sm_mhz"] = pclk.summary().get("sm_mhz")
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    nat.dgsm_set_profiling(True)
    with ClockSampler(gpu_index) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()   # L2 flushed between steps, outside the timed events
            starts[k].record(stream)
            sh = step(time_att=True)
            ends[k].record(stream)
            torch.cuda.synchronize()
            att_ms.append(ev_att[0].elapsed_time(ev_att[1]))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    prof = nat.dgsm_profile_collect()
    nat.dgsm_set_profiling(False)
    clocks = clk.summary()
    evals = stats["ray_evals"]
    from paper_2601_01660_b300 import shard
    total_ms, evals_all = shard.reduce_step_timing(float(sum(step_ms)), float(evals), device=dev)
    ms_per_step = total_ms / args.steps
    value = evals_all * args.steps / (total_ms * 1e-3)

    # ---- roofline of the dominant kernel (closed-form tile kernel) ----------
    tiles_ms = statistics.mean(p[1] for p in prof) if prof else None
    binning_ms = statistics.mean(p[0] for p in prof) if prof else None
    voxels = L * K * H * W
    shells = stats["shell_evals"]
    fp32 = FP32_PER_EVAL * evals + FP32_PER_SHELL * shells + FP32_PER_VOXEL * voxels
    n_ex2 = EX2_PER_EVAL * evals + EX2_PER_SHELL * shells + EX2_PER_VOXEL * voxels
    n_slow = RSQ_PER_EVAL * evals + RCP_PER_SHELL * shells      # rsqrt and rcp
    fp32_peak = peaks["fp32_ops_s"] / 1e12
    # MUFU: the op mix's rate when the pipe runs flat out on it
    mufu_ops = n_ex2 + n_slow
    mufu_peak = mufu_ops / (n_ex2 / peaks["ex2_ops_s"] + n_slow / peaks["rcp_ops_s"]) / 1e12
    fp32_ach = fp32 / (tiles_ms * 1e-3) / 1e12
    mufu_ach = mufu_ops / (tiles_ms * 1e-3) / 1e12
    if fp32_ach / fp32_peak >= mufu_ach / mufu_peak:
        bound_pipe, ach, peak = "fp32", fp32_ach, fp32_peak
    else:
        bound_pipe, ach, peak = "mufu", mufu_ach, mufu_peak
    traffic = _profiled_traffic(TILE_KERNEL, args.workload)
    roofline = {"bound": "alu", "kernel": TILE_KERNEL, "pipe": bound_pipe,
                "achieved": round(ach, 4), "peak": round(peak, 4), "unit": "Tops/s",
                "frac": round(ach / peak, 4), "traffic": traffic,
                "peak_source": "measured in this run (dgsm_measure_alu_peaks: FFMA and MUFU chains "
                               f"filling every SM, at {peaks.get('sm_mhz') or 'unsampled'} MHz), of measured",
                "work_per_unit": {"eval": f"{FP32_PER_EVAL} FP32 + rsqrt + ex2",
                                  "shell": f"{FP32_PER_SHELL} FP32 + rcp + ex2", "voxel": "1 FP32 + ex2"},
                "pipes": {"fp32": {"achieved": round(fp32_ach, 4), "peak": round(fp32_peak, 4),
                                   "frac": round(fp32_ach / fp32_peak, 4)},
                          "mufu": {"achieved": round(mufu_ach, 4), "peak": round(mufu_peak, 4),
                                   "frac": round(mufu_ach / mufu_peak, 4)}},
                "measured_peaks": {k: (round(v / 1e12, 3) if k.endswith("_s") else v) for k, v in peaks.items()},
                "kernel_ms": round(tiles_ms, 4),
                "ncu_pipe_utilisation": _profiled_pipes(TILE_KERNEL, args.workload)}

    # ---- attenuation roofline (HBM) -----------------------------------------
    # the event timer ticks in ~4 us steps on this part: the mean over steps
    # resolves a ~40 us kernel better than the median
    att = statistics.mean(att_ms)
    # algorithmic bytes: 36 per query (mean and colour read, colour written);
    # the atlas gathers hit a table the build has just written (L2-resident
    # in this step) and are reported apart
    att_bytes = N * 36
    hbm_peak = _measured_peak("hbm_gbs", 6400.0)
    attenuate = {"ms": round(att, 5), "gaussians_per_s": N / (att * 1e-3),
                 "achieved_gbs": round(att_bytes / (att * 1e-3) / 1e9, 1),
                 "peak_gbs": hbm_peak, "frac": round(att_bytes / (att * 1e-3) / 1e9 / hbm_peak, 4),
                 "algorithmic_bytes": att_bytes, "atlas_bytes": voxels * 4,
                 "gathers_per_query": 8 * L}
    # the paper's default receiver sampling: a Monte Carlo footprint of 8
    # points per Gaussian (timed on its own, after the steps, L2 flushed)
    fp_ms = []
    for k in range(5):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nat.dgsm_attenuate_footprint(atlas, radii, lights, means, quats, scales, colors, mode="mc",
                                     n_samples=8, seed=k, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            fp_ms.append(e0.elapsed_time(e1))
    fpt = statistics.mean(fp_ms)
    # receiver-driven region of interest around the avatar (Sec. 3.2): box
    # from the avatar, every scene Gaussian a receiver, the same atlas shape
    roi_ms = []
    box = torch.empty(5, dtype=torch.float32, device=dev)
    roi_atlas = torch.empty_like(atlas)
    nat.dgsm_set_profiling(True)
    for k in range(5):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nat.dgsm_roi_box(means[a0:a1], opac[a0:a1], R=2.0, z_margin=0.1, out=box)
        _, roi_mask, roi_k = nat.dgsm_build_roi(means, scales, quats, opac, lights, H, W, radii, means, box,
                                                out=roi_atlas, want_roi=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            roi_ms.append(e0.elapsed_time(e1))
    roi_prof = nat.dgsm_profile_collect()[2:]
    nat.dgsm_set_profiling(False)
    rk = roi_k.cpu().numpy()
    roi_vox = int(sum(int(roi_mask[l].sum().item()) * max(0, int(rk[l, 1]) - int(rk[l, 0]) + 1)
                      for l in range(L)))
    roi_t = statistics.mean(roi_ms)
    roi_st = nat.dgsm_get_build_stats()
    roi_tile_ms = statistics.mean(p[1] for p in roi_prof)
    # the region's tile kernel against the same FP32 roofline as the dense one
    # (its voxels outside P x [k_min, k_max] are written as 1 without work)
    roi_fp32 = (FP32_PER_EVAL * roi_st["ray_evals"] + FP32_PER_SHELL * roi_st["shell_evals"]
                + FP32_PER_VOXEL * roi_vox)
    roi_ach = roi_fp32 / (roi_tile_ms * 1e-3) / 1e12
    roi_build = {"ms": round(roi_t, 4), "box_half_width_m": 2.0, "voxels": roi_vox,
                 "phases_ms": {"prep_binning_sort": round(statistics.mean(p[0] for p in roi_prof), 4),
                               "tile_kernel": round(roi_tile_ms, 4)},
                 "ray_evals": int(roi_st["ray_evals"]),
                 "tile_kernel_roofline": {"bound": "alu", "pipe": "fp32", "achieved": round(roi_ach, 4),
                                          "peak": round(fp32_peak, 4), "unit": "Tops/s",
                                          "frac": round(roi_ach / fp32_peak, 4)},
                 "voxel_frac": round(roi_vox / voxels, 4), "dense_ms_per_build": None}
    # back-to-back calls: 20 calls captured in one CUDA graph (dgsm_graph) and
    # replayed between one event pair, so that neither the event resolution
    # nor the host's per-call time counts; at the workload's 1.6M receivers and
    # at 8x that many (positions repeated with millimetre offsets), whose 460 MB
    # of streamed inputs and outputs exceed L2
    def b2b(m, c):
        o = torch.empty_like(c)
        gs = torch.cuda.Stream(device=dev)
        for _ in range(3):
            nat.dgsm_attenuate(atlas, radii, lights, m, c, out=o)
        torch.cuda.synchronize()
        with nat.capture(gs) as cap:
            for _ in range(20):
                nat.dgsm_attenuate(atlas, radii, lights, m, c, out=o, stream=gs)
        g = cap.graph
        g.replay(gs)
        gs.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gs)
        g.replay(gs)
        e1.record(gs)
        torch.cuda.synchronize()
        g.close()
        ms = e0.elapsed_time(e1) / 20
        q = m.shape[0]
        return {"queries": q, "ms": round(ms, 5), "gaussians_per_s": q / (ms * 1e-3),
                "achieved_gbs": round(36 * q / (ms * 1e-3) / 1e9, 1),
                "frac": round(36 * q / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                "timing": "20 calls in one CUDA graph between one event pair"}
    attenuate["back_to_back"] = b2b(means, colors)
    attenuate["back_to_back_generated_order"] = b2b(t(sc0.means), t(sc0.colors))
    rep = 8
    big_m = (means.repeat(rep, 1) + 1e-3 * torch.arange(rep, device=dev, dtype=torch.float32)
             .repeat_interleave(N)[:, None]).contiguous()
    big_c = colors.repeat(rep, 1).contiguous()
    attenuate["large"] = b2b(big_m, big_c)
    del big_m, big_c
    attenuate["order"] = ("receivers stored in the z-order of their means (dgsm_spatial_order at load); "
                          "back_to_back_generated_order: the same receivers in the generator's random order")
    attenuate["bound"] = ("L1 (71% of its throughput) and issue (about 186 instructions per receiver); the Z-ordered atlas "
                          "taps hit L1 (0.9 L2 sectors per receiver); profiles/attenuate_room1p6m_x8.md")
    attenuate["footprint_mc8"] = {"ms": round(fpt, 5), "gaussians_per_s": N / (fpt * 1e-3),
                                  "achieved_gbs": round((N * 64) / (fpt * 1e-3) / 1e9, 1),
                                  "frac": round((N * 64) / (fpt * 1e-3) / 1e9 / hbm_peak, 4),
                                  "algorithmic_bytes": N * 64,
                                  "gathers_per_query": 8 * 8 * L}

    # ---- end to end through the host-buffer C entry point --------------------
    e2e = run_e2e(nat, wl, args, evals) if not args.no_e2e else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": step_config(wl, args.workload, world),
        "ms_per_build": round(statistics.mean(p[0] + p[1] for p in prof), 4) if prof else None,
        "build_phases_ms": {"prep_binning_sort": round(binning_ms, 4), "tile_kernel": round(tiles_ms, 4)},
        "attenuated_gaussians_per_s": attenuate["gaussians_per_s"],
        "attenuate": attenuate,
        "build_stats": stats,
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": None,
    }
    line["probe"] = time_probe(nat, sc, means, scales, quats, opac, colors, a0, a1, flush, stream, out)
    roi_build["dense_ms_per_build"] = line["ms_per_build"]
    if line["ms_per_build"]:
        roi_build["speedup_vs_dense"] = round(line["ms_per_build"] / roi_build["ms"], 3)
    line["roi_build"] = roi_build
    line["pca_normals"] = time_pca_normals(nat, means, quats, scales, opac, a0, a1, flush, stream)
    line["ablations"] = time_ablations(nat, (means, scales, quats, opac, colors), lights, radii, H, W,
                                       atlas, flush, stream)
    line["gpu_launches"] = count_launches(args, L)
    if rank == 0 and world == 1 and not args.no_reports:
        line.update(side_reports())
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, evals, args.cpu_texels)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def side_reports():
    """The precision, learned-surrogate and batched-frame reports, compact, so
    that the batched and learned forms are measured beside the plain form on
    the same GPU in the same run (the full reports: bench.py --report ...)."""
    import torch

    from paper_2601_01660_b300 import reports
    out = {}
    p = reports.precision()
    out["precision"] = {
        "workload": p["workload"],
        "max_abs_dT_vs_f32_store": {dt: [round(v["max"], 7) for v in p["abs_dT_vs_f32"][dt].values()]
                                    for dt in ("f16", "bf16")},
        "build_ms": p["build_ms"]}
    torch.cuda.empty_cache()
    s = reports.surrogate()
    out["surrogate"] = {
        "workload": s["workload"],
        "abs_dT_vs_exact": {k: {"p50": round(v["p50"], 6), "p99": round(v["p99"], 6)}
                            for k, v in s["abs_dT_vs_exact"].items()},
        "fallback_tile_fraction": {k: v for k, v in s["fallback_tile_fraction"].items() if k != "rule"},
        "memory_bytes": s["memory_bytes"],
        "gaussians_per_s": s["gaussians_per_s"],
        "training_s": s["training"]["seconds_total"]}
    torch.cuda.empty_cache()
    f = reports.frame()
    out["frame"] = {"workload": f["workload"], "ms_per_frame": f["ms_per_frame"],
                    "graph_nodes_per_frame": f["graph_nodes_per_frame"],
                    "persistent_graph_nodes_per_frame": f["persistent_graph_nodes_per_frame"],
                    "persistent_status": f["persistent_status"], "persistent_phase_ms": f["persistent_phase_ms"],
                    "stage_ms": f["stage_ms"], "chosen": f["chosen"]}
    torch.cuda.empty_cache()
    return out


def time_ablations(nat, gauss, lights, radii, H, W, atlas, flush, stream, F=208):
    """The ablation variants of Sec. 4 on the step's scene, each timed on its
    own (5 calls, the last 3 averaged, L2 flushed before each):
    (A) the 7-point stencil footprint (the 8-sample Monte Carlo one is in
    the line's attenuate);
    (B) the opacity-to-absorption mappings 1, 3 and 4 (the step builds with
    mapping 2, Eq. 5): build time and the pairs each one evaluates;
    (C) the cube-map atlas with about the octahedral atlas's texel count (six
    208 x 208 faces = 259,584 texels against 512^2 = 262,144): build time,
    attenuation through it, and how far its transmittances are from the
    octahedral atlas's at the receivers."""
    import torch
    means, scales, quats, opac, colors = gauss

    def timed(fn):
        ms = []
        for k in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= 2:
                ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    def build(params, h, w, out):
        nat.dgsm_set_profiling(True)
        t = timed(lambda k: nat.dgsm_build(means, scales, quats, opac, lights, h, w, radii, params=params,
                                           out=out))
        prof = nat.dgsm_profile_collect()[2:]
        nat.dgsm_set_profiling(False)
        st = nat.dgsm_get_build_stats()
        return {"ms": round(t, 4), "binning_ms": round(statistics.mean(p[0] for p in prof), 4),
                "tile_kernel_ms": round(statistics.mean(p[1] for p in prof), 4),
                "ray_evals": int(st["ray_evals"]), "evals_per_s": st["ray_evals"] / (t * 1e-3)}

    out = torch.empty_like(colors)
    res = {"footprint_stencil7_ms": round(timed(lambda k: nat.dgsm_attenuate_footprint(
        atlas, radii, lights, means, quats, scales, colors, mode="stencil7", out=out)), 5)}
    tmp = torch.empty_like(atlas)
    res["beta_mode"] = {str(m): build({"beta_mode": m}, H, W, tmp) for m in (1, 3, 4)}
    L, K = atlas.shape[0], atlas.shape[1]
    cube = torch.empty((L, K, 6 * F, F), dtype=torch.float32, device=atlas.device)
    c = build({"atlas_map": 1}, 6 * F, F, cube)
    c.update({"face": F, "texels": 6 * F * F, "octahedral_texels": H * W})
    c["attenuate_ms"] = round(timed(lambda k: nat.dgsm_attenuate_cube(cube, radii, lights, means, colors,
                                                                      out=out)), 5)
    nat.dgsm_build(means, scales, quats, opac, lights, H, W, radii, out=tmp)
    _, To = nat.dgsm_attenuate(tmp, radii, lights, means, colors, want_T=True)
    _, Tc = nat.dgsm_attenuate_cube(cube, radii, lights, means, colors, want_T=True)
    dT = (To - Tc).abs().flatten()
    c["T_vs_octahedral"] = {"mean_abs": round(dT.mean().item(), 6),
                            "p99_abs": round(torch.quantile(dT[::max(1, dT.numel() // 1000000)].float(),
                                                            0.99).item(), 6)}
    res["cube_map"] = c
    return res


def time_pca_normals(nat, means, quats, scales, opac, a0, a1, flush, stream, radius=0.05):
    """Local-PCA pseudo-normals (Sec. 4) of the avatar (its own Gaussians as
    neighbours, oriented away from its centroid) and of the whole room, r =
    5 cm; L2 flushed before each timed call."""
    import torch
    out = {"radius_m": radius}
    cen = nat.dgsm_weighted_centroid(means[a0:a1], opac[a0:a1])
    for name, sl in (("avatar", slice(a0, a1)), ("room", slice(0, means.shape[0]))):
        m, q, s, o = means[sl], quats[sl], scales[sl], opac[sl]
        res = torch.empty_like(m)
        ms = []
        for k in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nat.dgsm_pca_normals(m, o, q, s, cen, radius=radius, out=res)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= 2:
                ms.append(e0.elapsed_time(e1))
        t = statistics.mean(ms)
        out[name] = {"gaussians": int(m.shape[0]), "ms": round(t, 4),
                     "gaussians_per_s": m.shape[0] / (t * 1e-3)}
    return out


def time_probe(nat, sc, means, scales, quats, opac, colors, a0, a1, flush, stream, final):
    """The cubemap probe of Sec. 3.4 at the avatar: the room without its
    avatar splatted on six 64x64 faces at the avatar's alpha-weighted
    centroid, then the SH fit of the rendered radiance (timed apart from the
    step, L2 flushed, mean of 3 after 2 warm-up calls)."""
    import torch
    face = 64
    keep = torch.cat([torch.arange(0, a0), torch.arange(a1, sc.n)]).to(means.device)
    sm, ss, sq, so, scol = (t.index_select(0, keep).contiguous() for t in (means, scales, quats, opac, colors))
    dirs, w = nat.dgsm_cube_dirs(face)
    rgb = torch.empty((6 * face * face, 3), dtype=torch.float32, device=means.device)
    ms_r, ms_f = [], []
    pairs = 0
    for k in range(5):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        cen = nat.dgsm_weighted_centroid(means[a0:a1], opac[a0:a1])
        _, pairs = nat.dgsm_render_cubemap(sm, ss, sq, so, scol, cen, face=face, out=rgb, want_pairs=True)
        e1.record(stream)
        nat.sh_fit(dirs, rgb, w)
        e2.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            ms_r.append(e0.elapsed_time(e1))
            ms_f.append(e1.elapsed_time(e2))
    probe = {"face": face, "scene_gaussians": int(keep.numel()), "splat_pairs": int(pairs),
             "render_ms": round(statistics.mean(ms_r), 4), "sh_fit_ms": round(statistics.mean(ms_f), 4),
             "mean_radiance": [round(float(x), 4) for x in rgb.mean(0).tolist()]}
    # the final composite: every Gaussian (scene and avatar, the step's
    # attenuated and relit colours) seen from 3 m at 1280 x 720
    from paper_2601_01660_b300 import scenes
    W, H = 1280, 720
    cam = torch.as_tensor(scenes.look_at_camera([-1.2, -1.5, 1.6], [1.5, 0.0, 0.9], W, H, 60.0))[None].to(means.device)
    img = torch.empty((1, H, W, 3), dtype=torch.float32, device=means.device)
    ms_c = []
    for k in range(5):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, cpairs = nat.dgsm_render_views(means, scales, quats, opac, final, cam, W, H, out=img, want_pairs=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            ms_c.append(e0.elapsed_time(e1))
    probe["composite"] = {"width": W, "height": H, "gaussians": int(sc.n), "splat_pairs": int(cpairs),
                          "render_ms": round(statistics.mean(ms_c), 4)}
    return probe


def count_launches(args, L):
    """Kernels of ours per step.  Build with at most 64 super-tiles per light
    (the room's 512 x 512 atlas): cones 1, prep 1, super-tile count 1, scan 3,
    keep 1, key ranges 1, super-tile scatter 1, unit count 1, scan 3, unit
    fill 1, tile count 1, scan 3, keep 1, tile emit 1, tile ranges 1, item
    count 1, scan 3, item expand 1, tile kernel 1 (27); with more super-tiles
    the sorted lists of dgsm_bin instead: super-tile count 1, scan 3, keep 1,
    super-tile emit 1, sort passes x (hist 1 + scan 3 + scatter 1), super-tile
    ranges 1.  Then attenuate 1, sh_fit 2, centroid 2, relight 1."""
    import math
    per_light = math.ceil(512 / 8 / 8) ** 2
    if per_light <= 64:
        build = 27
    else:
        sort_passes = math.ceil(max(1, (per_light * L - 1).bit_length()) / 8)
        build = 27 + 5 * sort_passes
    return (build + 6) * args.steps


def _tile_kernel_sha():
    """sha256 of the tile kernel's own source: its device code in
    build_device.cuh (from the closed-form helpers to the end of the file)
    and its __global__ wrapper in build.cu, so that edits elsewhere keep a
    profile of it valid."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2601_01660_b300", "csrc")
    dev = open(os.path.join(csrc, "build_device.cuh")).read()
    bu = open(os.path.join(csrc, "build.cu")).read()
    b0 = bu.index("build_tiles_kernel(")
    b1 = bu.index("\n}\n", b0)
    return hashlib.sha256((dev[dev.index("// erfc(y) for y >= 0"):] + bu[b0:b1]).encode()).hexdigest()


def _profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of this
    workload, or None when the summary is missing or was taken on another
    version of the kernel source (its sha256 is recorded beside the figure)."""
    path = os.path.join(ROOT, "profiles", f"{kernel.replace('_kernel', '')}_{workload}.txt")
    try:
        fields = dict(line.split(":", 1) for line in open(path) if ":" in line)
        if fields.get("source_sha256", "").strip() != _tile_kernel_sha():
            return None
        return int(fields["dram_bytes_per_launch"].strip())
    except (OSError, KeyError, ValueError):
        return None


def _profiled_pipes(kernel, workload):
    """ncu pipe utilisation (fraction of peak over active cycles) of `kernel`
    from the full capture summarised beside its traffic figure, under the same
    source-hash rule, or None."""
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel.replace('_kernel', '')}_{workload}.txt")
    try:
        text = open(path).read()
        if f"source_sha256: {_tile_kernel_sha()}" not in text:
            return None
        m = re.search(r"FMA ([0-9.]+)%, ALU ([0-9.]+)%,(?: LSU [0-9.]+%,)? XU \(MUFU\) ([0-9.]+)%", text)
        if not m:
            return None
        return {"fma": float(m.group(1)) / 100, "alu": float(m.group(2)) / 100,
                "xu": float(m.group(3)) / 100,
                "source": f"ncu --set full on the room550k case (profiles/{kernel.replace('_kernel', '')}_room1p6m.txt)"}
    except (OSError, ValueError):
        return None


def _measured_peak(key, fallback):
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except (OSError, KeyError, ValueError):
        return fallback


def run_e2e(nat, wl, args, evals):
    """The step through the public host-buffer API: every step copies its
    inputs from pinned host memory and its colours and SH back.  Timed two
    ways: frames submitted to the two slots of a FrameQueue in turn (frame
    f's compute overlaps frame f + 1's copy-in and frame f - 1's copy-out;
    the line's value), and one blocking dgsm_frame_host call per step."""
    import torch
    sc = wl["occluders"]
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    h = {k: pin(getattr(sc, k)) for k in ("means", "scales", "quats", "opac", "colors")}
    D, Y, w = (pin(a) for a in wl["cubemap"])
    lights, radii = pin(wl["lights"]), pin(wl["radii"])
    sl = sc.meta["avatar"]
    outs = [(torch.empty((sc.n, 3), dtype=torch.float32).pin_memory(),
             torch.empty((3, 9), dtype=torch.float32).pin_memory()) for _ in range(2)]
    args_in = (h["means"], h["scales"], h["quats"], h["opac"], h["colors"], lights, wl["H"], wl["W"], radii, D, Y, w)
    call = lambda: nat.dgsm_frame_host(*args_in, relight_range=(sl.start, sl.stop), colors_out=outs[0][0],
                                       sh_out=outs[0][1])
    q = nat.FrameQueue()
    submit = lambda f: q.submit(*args_in, relight_range=(sl.start, sl.stop), colors_out=outs[f % 2][0],
                                sh_out=outs[f % 2][1])
    n = max(3, min(args.steps, 20))
    for _ in range(max(1, args.warmup)):
        call()
    for f in range(2):
        q.wait(submit(f))
    torch.cuda.synchronize()
    # pipelined: n frames, each submitted before the previous one is waited for
    t0 = time.perf_counter()
    slots = [submit(0)]
    for f in range(1, n):
        slots.append(submit(f))
        q.wait(slots[f - 1])
    q.wait(slots[-1])
    dt = (time.perf_counter() - t0) / n
    # blocking: one call per step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        call()
    dt_block = (time.perf_counter() - t0) / n
    h2d = sum(t.numel() * 4 for t in h.values()) + (D.numel() + Y.numel() + w.numel()
                                                    + lights.numel() + radii.numel()) * 4
    d2h = outs[0][0].numel() * 4 + outs[0][1].numel() * 4
    return {"value": evals / dt, "unit": UNIT, "ms_per_step": round(dt * 1e3, 4),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": "FrameQueue (dgsm_frame_host_submit / _wait, two slots; host buffers, pinned)",
            "blocking": {"value": evals / dt_block, "ms_per_step": round(dt_block * 1e3, 4),
                         "api": "dgsm_frame_host (one blocking call per step)"}}


# ----------------------------------------------------------------------------- oracle

def oracle_step(wl, lij, q_idx, r_idx, atlas=None):
    """One bounded sample of the step on the FP64 oracle, extrapolated to the
    whole step: the build at texels lij (its per-call setup over every
    Gaussian timed alone, with no texel, so that it counts once; the texels,
    a whole number of waves of the oracle's threads, give the per-texel cost
    for every texel), attenuation of queries q_idx (scaled to every
    receiver), the full SH fit, relight of avatar Gaussians r_idx (scaled to
    the whole avatar).  `atlas` is an all-ones array of the atlas shape,
    allocated outside the timing; it is restored before return.  Returns
    (full-step seconds, seconds the sample took)."""
    import oracle
    from paper_2601_01660_b300 import scenes
    sc, lights, radii, H, W = wl["occluders"], wl["lights"], wl["radii"], wl["H"], wl["W"]
    L, K = lights.shape[0], radii.shape[0]
    if atlas is None:
        atlas = np.ones((L, K, H, W))
    n = lij.shape[0]
    t0 = time.perf_counter()
    oracle.build_tau_texels(sc, lights, H, W, radii, lij[:0])
    t1 = time.perf_counter()
    tau = oracle.build_tau_texels(sc, lights, H, W, radii, lij)
    t2 = time.perf_counter()
    setup = t1 - t0
    per_texel = max((t2 - t1) - setup, 0.0) / max(n, 1)
    build_full = setup + per_texel * L * H * W
    # attenuate the sampled queries against an atlas that holds the sampled texels
    atlas[lij[:, 0], :, lij[:, 1], lij[:, 2]] = np.exp(-tau)
    q = scenes.subset(sc, q_idx)
    t3 = time.perf_counter()
    oracle.attenuate(atlas, radii, lights, q.means, q.colors)
    t4 = time.perf_counter()
    atlas[lij[:, 0], :, lij[:, 1], lij[:, 2]] = 1.0
    D, Y, w = wl["cubemap"]
    shc = oracle.sh_fit(D, Y, w)
    t5 = time.perf_counter()
    av = scenes.subset(sc, r_idx)
    oracle.relight(shc, av, av.means.astype(np.float64).mean(0))
    t6 = time.perf_counter()
    sl = sc.meta["avatar"]
    full = (build_full + (t4 - t3) * sc.n / max(q_idx.size, 1) + (t5 - t4)
            + (t6 - t5) * (sl.stop - sl.start) / max(r_idx.size, 1))
    return full, t6 - t0


def _oracle_sample(wl, n_texels, seed=0):
    """Random texels (a whole number of waves of the oracle's threads, so the
    timed sample keeps every core busy as the full build would), and matching
    fractions of the receivers and of the avatar."""
    import oracle
    cores = max(1, oracle.num_threads())
    n_texels = -(-max(n_texels, cores) // cores) * cores
    rng = np.random.default_rng(seed)
    sc = wl["occluders"]
    H, W, L = wl["H"], wl["W"], wl["lights"].shape[0]
    flat = rng.choice(L * H * W, size=n_texels, replace=False)
    l, rem = np.divmod(flat, H * W)
    lij = np.stack([l, rem // W, rem % W], 1).astype(np.int32)
    frac = n_texels / (L * H * W)
    n_q = max(1, int(round(frac * sc.n)))
    sl = sc.meta["avatar"]
    n_r = max(1, int(round(frac * (sl.stop - sl.start))))
    q_idx = rng.choice(sc.n, size=n_q, replace=False)
    r_idx = sl.start + rng.choice(sl.stop - sl.start, size=n_r, replace=False)
    return lij, q_idx, r_idx, frac


def _oracle_eval_count(wl, stride=16):
    """Gaussian-ray evaluations of the whole build, estimated on the oracle
    from a regular grid of texels (every stride-th row and column of every
    light's atlas): counting is far cheaper than evaluating, so the count's
    sample can be much larger than the timed one."""
    import oracle
    H, W, L = wl["H"], wl["W"], wl["lights"].shape[0]
    ii, jj = np.meshgrid(np.arange(stride // 2, H, stride), np.arange(stride // 2, W, stride), indexing="ij")
    lij = np.concatenate([np.stack([np.full(ii.size, l), ii.ravel(), jj.ravel()], 1) for l in range(L)])
    lij = lij.astype(np.int32)
    n = oracle.count_ray_evals(wl["occluders"], wl["lights"], H, W, wl["radii"], lij)
    return n * (L * H * W) / lij.shape[0], lij.shape[0]


def cpu_baseline(wl, evals_full, n_texels):
    """The oracle (FP64 brute force, OpenMP on the host cores) on a bounded
    sample of the step, scaled to the metric's unit."""
    import oracle
    lij, q_idx, r_idx, frac = _oracle_sample(wl, n_texels)
    n_texels = lij.shape[0]
    t_full, t_sample = oracle_step(wl, lij, q_idx, r_idx)
    evals_est, n_count = _oracle_eval_count(wl)
    value = evals_est / t_full
    return {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"{n_texels} random texels of the 512x512x64 build x all 1.6M Gaussians x 64 "
                       f"shells (setup and per-texel cost timed apart), {q_idx.size} attenuated "
                       f"queries, {r_idx.size} relit avatar Gaussians, full SH fit; each part "
                       f"extrapolated to the full step ({t_full:.0f} s); the step's "
                       f"Gaussian-ray evals ({evals_est:.3g}) counted by the oracle on a "
                       f"{n_count}-texel grid"),
            "sample_seconds": round(t_sample, 2), "evals_full_gpu_count": int(evals_full)}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one bounded sample."""
    if rank != 0:
        return
    import oracle
    wl = load_workload(0)
    # keep the whole --steps/--warmup run to a couple of minutes
    # as many waves of the oracle's threads per step (1 to 4) as keep the
    # timed steps near 150 s: one wave, timed once here, sets the pace (a
    # single wave runs at the pace of its slowest thread, so more waves
    # measure the build's per-texel cost more fairly)
    cores = max(1, oracle.num_threads())
    lij1, _, _, _ = _oracle_sample(wl, cores)
    t0 = time.perf_counter()
    oracle.build_tau_texels(wl["occluders"], wl["lights"], wl["H"], wl["W"], wl["radii"], lij1)
    t_wave = max(time.perf_counter() - t0, 1e-3)
    waves = int(min(4, max(1, 150.0 / (max(1, args.steps) * t_wave))))
    lij, q_idx, r_idx, frac = _oracle_sample(wl, waves * cores)
    n_tex = lij.shape[0]
    evals_est, n_count = _oracle_eval_count(wl)
    atlas = np.ones((wl["lights"].shape[0], wl["radii"].shape[0], wl["H"], wl["W"]))
    for _ in range(args.warmup):
        oracle_step(wl, lij[:0], q_idx[:1], r_idx[:1], atlas)
    runs = [oracle_step(wl, lij, q_idx, r_idx, atlas) for _ in range(args.steps)]
    t_full = statistics.mean(r[0] for r in runs)      # the whole step, extrapolated from the sample
    t_sample = statistics.mean(r[1] for r in runs)    # what each timed step took
    value = evals_est / t_full
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_sample * 1e3, 1),
            "full_step_s_extrapolated": round(t_full, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": step_config(wl, WORKLOAD, world),
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": value,
                             "sample": (f"{n_tex} random texels of the 512x512x64 build x all "
                                        f"Gaussians x 64 shells per step (setup and per-texel cost "
                                        f"timed apart), matching fractions of the attenuation and "
                                        f"relight, full SH fit; each part extrapolated; the step's "
                                        f"evals counted by the oracle on a {n_count}-texel grid")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["room1p6m", "room550k"], default=WORKLOAD,
                    help="room550k: the same room at a third of the size (profiler captures)")
    ap.add_argument("--cpu-texels", type=int, default=72)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-reports", action="store_true",
                    help="leave out the precision, surrogate and frame reports of the line")
    ap.add_argument("--frame-workload", choices=["crowd8", "crowd8s"], default="crowd8",
                    help="the frame report's workload (crowd8s: a tenth of the Gaussians, for profiler captures)")
    ap.add_argument("--report", choices=["precision", "surrogate", "frame", "field"],
                    help="print a side report (one JSON line) instead of the step benchmark")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = _env_rank()
    if args.report:
        from paper_2601_01660_b300 import reports
        reports.main(args.report, frame_workload=args.frame_workload)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
