// frame_kernel.cu -- the moving-avatar frame (Secs. 3.2-3.5) as one
// persistent cooperative kernel.
//
// Every block of the launch stays resident for the whole frame (a
// cooperative launch guarantees that they all run at once), and the
// frame's steps are separated by grid-wide barriers instead of kernel
// boundaries:
//
//   P1  per (light, avatar Gaussian): rigid motion to this frame's pose,
//       the prep (the build record, and the binning record's super-tile cone
//       tests as a bit mask), counted per (light, super-tile) key; per-object
//       centroid partial sums
//   B1
//   P2  block 0: key offsets, fine-binning units, the centroids
//   B2
//   P3  super-tile lists: every (light, Gaussian) writes itself into the
//       lists of the super-tiles it reaches (ranges reserved per block and key)
//   B3
//   P4  fine binning, one unit (<= 512 Gaussians of one list) per block at a
//       time: the binning records formed anew from the rest pose, cone and
//       ellipsoid tests against the 64 tiles, per-tile counts
//   B4
//   P5  block 0: tile offsets and the tiles' work items
//   B5
//   P6  per-tile lists written from the fine bitmaps (per-tile cursors)
//   B6
//   P7  the closed-form accumulation of the dynamic atlases (the build's
//       tile worker: blocks pull work items from a counter)
//   B7
//   P8  every receiver attenuated by the static and dynamic atlases; the
//       avatar receivers then relit around their object's centroid
//
// Barrier waits are bounded (clock64 budget); a block that gives up records
// DGSM_ERR_TIMEOUT, raises the abort flag and returns, and every other block
// returns at its next barrier.  The per-voxel accumulators of P7 are only
// touched by blocks that passed B6, which then consume every work item, so
// they are back to zero whatever barrier failed.
//
// The arithmetic of every step is that of the standalone kernels (shared
// device functions), so the frame equals the separate calls up to the order
// of the floating-point atomic sums in the atlas.  Lists come out in an
// order set by atomics rather than sorted; each tile's sum does not depend
// on it beyond rounding.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "build_device.cuh"
#include "lookup.cuh"
#include "motion.cuh"
#include "relight.cuh"

namespace dgsm {
namespace {

constexpr int FR_THREADS = 256;
constexpr int FR_MIN_BLOCKS = 4;     // resident blocks per SM the register budget targets
constexpr int FR_MAX_SKEYS = 4096;   // lights x super-tiles (the per-block histogram of P1)
constexpr int FR_MAX_TKEYS = 65536;  // lights x tiles
constexpr int FR_TAB = 1024;         // relight directions in shared memory at a time
constexpr int FR_RG = 3;             // avatar receivers per relight group of a thread
constexpr int FR_ATT_U = 2;          // static receivers in flight per thread (1, 3, 4, 8 measured slower)
constexpr long long FR_BUDGET = 4000000000ll;  // cycles a barrier waits (about 2 s)

// Control words, zeroed before every launch.
struct FrameCtl {
    unsigned bar_count, bar_gen, abort, item_counter;
    unsigned skip, done_blocks, unit_counter, emit_counter;  // counters of P4 and P6
    unsigned long long n_units, n_items;
};

struct FrameDev {
    // receivers: [0, n_static) static, then the avatars
    const float *q_means;  // static rows are read
    const float *cin;
    float *cout;
    int64_t n_static;
    // static atlases, float32 [L][K][H][W]
    const float *sat;
    int H, W, K;
    const float *radii;
    // avatars
    const float *rest_means, *rest_quats, *scales, *opac;
    float *av_means, *av_quats;  // written (the frame's moved Gaussians)
    int64_t N;
    const float *poses;  // device copy, n_obj x 8
    // dynamic atlases, float32 [L][Kd][Hd][Wd], tile 8
    float *dyn;
    int Hd, Wd, Kd;
    const float *radii_d;
    int tx, ty, sx, n_tiles, n_super;
    const float *lights;
    int L;
    float kappa, eps_cull, wd;
    int beta_mode, chunk;
    // relight
    const float *sh;
    float rq, rgamma, rt_max, reps;
    int nth, nph;
    float *centroids;
    int cen_bps;
    // workspace
    const float4 *cones;
    BuildRec *brec;
    unsigned long long *smask;         // [L N] super-tiles each (light, Gaussian) reaches (n_super <= 64)
    uint32_t *skey_cnt, *skey_cur, *skey_start, *unit_off;  // [L n_super]
    uint32_t *cvals;                   // [capC]
    Unit *units;                       // [max_units]
    uint32_t *fcnt, *fmask;            // [max_units][64], [max_units][64][3][MASK_WORDS]
    uint32_t *tile_cnt, *ts, *te, *tcur, *item_off;  // [L n_tiles]
    Item *items;                       // [max_items]
    uint32_t *vals;                    // [cap]
    float *accum;
    unsigned *done;
    double *cen_part;
    FrameCtl *ctl;
    int *status;
    unsigned long long *stats;
    uint32_t capC, cap, max_units, max_items;
    int timeout_barrier;
    unsigned long long *phase_ns;  // nullptr, or 9 timestamps: start, each barrier, end
    Segs segs;
};

// Grid-wide barrier `idx` (1-based).  Thread 0 of each block arrives on a
// counter; the last arrival resets it and advances the generation, the
// others wait for the generation to move, for at most FR_BUDGET cycles.
// Returns false (in every thread of the block) when the frame is aborted.
__device__ __noinline__ bool grid_sync(const FrameDev &d, int idx) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        FrameCtl *c = d.ctl;
        volatile unsigned *vgen = &c->bar_gen, *vabort = &c->abort;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else if (idx != d.timeout_barrier) {
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (*vabort) { ok = 0; break; }
                if (clock64() - t0 > FR_BUDGET) {
                    atomicExch(&c->abort, 1u);
                    record_status(d.status, DGSM_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (idx == d.timeout_barrier) {
            // the failure path on request: every block gives up here
            atomicExch(&c->abort, 1u);
            record_status(d.status, DGSM_ERR_TIMEOUT);
            ok = 0;
        }
        __threadfence();
        if (*vabort) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Phase timing (when the context profiles): block 0 stamps the global timer
// at the start and as it leaves each barrier; the last block to finish
// stamps the end.
__device__ __forceinline__ void stamp(const FrameDev &d, int k) {
    if (d.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        d.phase_ns[k] = t;
    }
}

// Per-block tables of the attenuation (both atlases' radii and shell-guess
// tables, the lights and their weights), carved from shared memory.
struct AttTabs {
    float *rs, *inw, *rsd, *inwd, *ls, *wl;
    short *tab, *tabd;
    ShellTab st, std_;
};
constexpr size_t ATT_TAB_BYTES = sizeof(float) * (4 * 256 + 64 * 3 + 64) + sizeof(short) * 2 * SHELL_BINS;

__device__ __forceinline__ AttTabs att_tabs(const FrameDev &d, void *base) {
    AttTabs a;
    float *f = (float *)base;
    a.rs = f; a.inw = f + 256; a.rsd = f + 512; a.inwd = f + 768; a.ls = f + 1024; a.wl = f + 1024 + 192;
    a.tab = (short *)(f + 1024 + 256);
    a.tabd = a.tab + SHELL_BINS;
    for (int k = threadIdx.x; k < d.K; k += blockDim.x) {
        a.rs[k] = d.radii[k];
        a.inw[k] = k + 1 < d.K ? 1.0f / (d.radii[k + 1] - d.radii[k]) : 0.0f;
    }
    for (int k = threadIdx.x; k < d.Kd; k += blockDim.x) {
        a.rsd[k] = d.radii_d[k];
        a.inwd[k] = k + 1 < d.Kd ? 1.0f / (d.radii_d[k + 1] - d.radii_d[k]) : 0.0f;
    }
    for (int k = threadIdx.x; k < 3 * d.L; k += blockDim.x) a.ls[k] = d.lights[k];
    for (int k = threadIdx.x; k < d.L; k += blockDim.x) a.wl[k] = 1.0f / (float)d.L;
    __syncthreads();
    a.st = build_shell_tab(a.rs, d.K, a.tab);
    a.std_ = build_shell_tab(a.rsd, d.Kd, a.tabd);
    __syncthreads();
    return a;
}

// acc[u] = sum_l w_l T_static,l(p_u) T_dyn,l(p_u) for U receivers at once,
// the lights outside so that their gathers are in flight together (as in
// dgsm_attenuate_dyn, with the same arithmetic per receiver).  The dynamic
// atlases were written by this kernel: their taps are read through L2.
template <int U>
__device__ __forceinline__ void att_batch(const FrameDev &d, const AttTabs &at, const float (&px)[U],
                                          const float (&py)[U], const float (&pz)[U], float (&acc)[U]) {
    const uint32_t lstride = (uint32_t)d.K * d.H * d.W, dstride = (uint32_t)d.Kd * d.Hd * d.Wd;
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0f;
    for (int l = 0; l < d.L; ++l) {
        const float ox = at.ls[3 * l], oy = at.ls[3 * l + 1], oz = at.ls[3 * l + 2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const SampleIndex s = sample_index_tab(px[u], py[u], pz[u], ox, oy, oz, d.H, d.W, at.rs, d.K, at.tab, at.st);
            float Tl = 1.0f;
            if (s.t != 0.0f) {
                Tl = lookup<float>(d.sat + (size_t)l * lstride, d.H, d.W, d.K, s, at.rs, at.inw);
                const SampleIndex sd =
                    sample_index_tab(px[u], py[u], pz[u], ox, oy, oz, d.Hd, d.Wd, at.rsd, d.Kd, at.tabd, at.std_);
                Tl *= lookup<float, true>(d.dyn + (size_t)l * dstride, d.Hd, d.Wd, d.Kd, sd, at.rsd, at.inwd);
            }
            acc[u] = fmaf(at.wl[l], Tl, acc[u]);
        }
    }
}

// The binning record of avatar Gaussian g for light l, formed anew from its
// rest pose and this frame's motion (the same floats as the prep's).
__device__ __forceinline__ BinRec frame_binrec(const FrameDev &d, const float (*pose)[16], int l, int64_t g) {
    const float *r = pose[d.segs.n == 1 ? 0 : seg_find(d.segs, g)];
    const float3 m = pose_point(r, d.rest_means[3 * g], d.rest_means[3 * g + 1], d.rest_means[3 * g + 2]);
    const float4 q = pose_quat(r, reinterpret_cast<const float4 *>(d.rest_quats)[g]);
    BinRec br;
    prep_core((int64_t)l * d.N + g, l, m.x, m.y, m.z, d.scales[3 * g], d.scales[3 * g + 1], d.scales[3 * g + 2], q.x,
              q.y, q.z, q.w, d.opac[g], d.lights[3 * l], d.lights[3 * l + 1], d.lights[3 * l + 2], d.radii_d, d.Kd,
              d.kappa, d.eps_cull, nullptr, br, d.status, nullptr, d.beta_mode);
    return br;
}

// Super-tiles reached by (light l, Gaussian g) as a bit mask (n_super <= 64).
__device__ __forceinline__ unsigned long long super_mask(const FrameDev &d, const BinRec &br) {
    const int mode = (int)br.b.y;
    unsigned long long m = 0ull;
    if (mode == 0) return m;
    const float4 *scones = d.cones + 2 * d.n_tiles;
    for (int sidx = 0; sidx < d.n_super; ++sidx)
        if (mode == 2 || cone_overlap(br, scones + 2 * sidx)) m |= 1ull << sidx;
    return m;
}

// Exclusive scan over n entries (one block; every thread calls it): get(i)
// gives entry i, put(i, prefix, value) receives its exclusive prefix.
// Thread t takes a contiguous run of entries.  Returns the 64-bit total.
template <typename Get, typename Put>
__device__ __forceinline__ unsigned long long block_scan(int n, Get get, Put put, unsigned long long *s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + FR_THREADS - 1) / FR_THREADS;
    const int b = min(tid * per, n), e = min(b + per, n);
    unsigned long long local = 0;
    for (int i = b; i < e; ++i) local += get(i);
    unsigned long long x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = lane < FR_THREADS / 32 ? s_warp[lane] : 0ull;
        for (int o = 1; o < FR_THREADS / 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULLMASK, v, o);
            if (lane >= o) v += y;
        }
        if (lane < FR_THREADS / 32) s_warp[lane] = v;
    }
    __syncthreads();
    unsigned long long run = x - local + (warp ? s_warp[warp - 1] : 0ull);
    for (int i = b; i < e; ++i) {
        const uint32_t c = get(i);
        put(i, run, c);
        run += c;
    }
    const unsigned long long total = s_warp[FR_THREADS / 32 - 1];
    __syncthreads();
    return total;
}

__device__ __forceinline__ Unit load_unit(const Unit *u) {
    const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(u)), b = __ldcg(reinterpret_cast<const uint4 *>(u) + 1);
    Unit U;
    U.key = a.x; U.start = a.y; U.end = a.z; U.ju = a.w;
    U.u0 = b.x; U.pad0 = b.y; U.pad1 = b.z; U.pad2 = b.w;
    return U;
}

// Shared memory of the phases (one dynamic buffer, reused phase after phase).
__host__ __device__ constexpr size_t relight_smem_bytes() {
    return ATT_TAB_BYTES + sizeof(float4) * 2 * FR_TAB + sizeof(float) * (28 + 3 * MAX_OBJECTS);
}

__global__ void __launch_bounds__(FR_THREADS, FR_MIN_BLOCKS) crowd_frame_kernel(const __grid_constant__ FrameDev d) {
    extern __shared__ float4 fsm[];
    __shared__ float s_pose[MAX_OBJECTS][16];
    __shared__ double s_red[FR_THREADS / 32][4];
    __shared__ unsigned long long s_warp[FR_THREADS / 32];
    __shared__ unsigned s_next;  // the unit a block takes next (P4, P6)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t gtid = (int64_t)blockIdx.x * FR_THREADS + tid, gstride = (int64_t)gridDim.x * FR_THREADS;
    const int64_t N = d.N;
    const int nsk = d.L * d.n_super, ntk = d.L * d.n_tiles;
    stamp(d, 0);
    for (int o = tid; o < d.segs.n; o += FR_THREADS) pose_matrix(d.poses + 8 * o, s_pose[o]);
    __syncthreads();

    // ---- P1: motion, prep, super-tile counts, centroid partial sums ----
    {
        const int nv = d.segs.n * d.cen_bps;
        for (int vb = blockIdx.x; vb < nv; vb += gridDim.x) {
            const int o = vb / d.cen_bps;
            const float *r = s_pose[o];
            const float *rm = d.rest_means;
            centroid_partial_block(
                d.opac, d.segs, o, vb - o * d.cen_bps, d.cen_bps,
                [&](long long i) { return pose_point(r, rm[3 * i], rm[3 * i + 1], rm[3 * i + 2]); }, d.cen_part,
                s_red);
        }
        uint32_t *hist = reinterpret_cast<uint32_t *>(fsm);  // [nsk]
        for (int k = tid; k < nsk; k += FR_THREADS) hist[k] = 0u;
        __syncthreads();
        const int64_t total = (int64_t)d.L * N;
        const float4 *scones = d.cones + 2 * d.n_tiles;
        for (int64_t idx = gtid; idx < total; idx += gstride) {
            const int l = (int)(idx / N);
            const int64_t g = idx - (int64_t)l * N;
            const float *r = s_pose[d.segs.n == 1 ? 0 : seg_find(d.segs, g)];
            const float3 m = pose_point(r, d.rest_means[3 * g], d.rest_means[3 * g + 1], d.rest_means[3 * g + 2]);
            const float4 q = pose_quat(r, reinterpret_cast<const float4 *>(d.rest_quats)[g]);
            if (l == 0) {
                d.av_means[3 * g] = m.x;
                d.av_means[3 * g + 1] = m.y;
                d.av_means[3 * g + 2] = m.z;
                reinterpret_cast<float4 *>(d.av_quats)[g] = q;
            }
            BinRec br;
            prep_core(idx, l, m.x, m.y, m.z, d.scales[3 * g], d.scales[3 * g + 1], d.scales[3 * g + 2], q.x, q.y,
                      q.z, q.w, d.opac[g], d.lights[3 * l], d.lights[3 * l + 1], d.lights[3 * l + 2], d.radii_d,
                      d.Kd, d.kappa, d.eps_cull, d.brec, br, d.status, nullptr, d.beta_mode);
            if (d.n_super <= 64) {
                unsigned long long sm = super_mask(d, br);
                d.smask[idx] = sm;
                for (; sm; sm &= sm - 1) atomicAdd(&hist[l * d.n_super + __ffsll(sm) - 1], 1u);
            } else {
                const int mode = (int)br.b.y;
                if (mode != 0)
                    for (int sidx = 0; sidx < d.n_super; ++sidx)
                        if (mode == 2 || cone_overlap(br, scones + 2 * sidx)) atomicAdd(&hist[l * d.n_super + sidx], 1u);
            }
        }
        __syncthreads();
        for (int k = tid; k < nsk; k += FR_THREADS) {
            const uint32_t c = hist[k];
            if (c) atomicAdd(d.skey_cnt + k, c);
        }
    }
    if (!grid_sync(d, 1)) return;
    stamp(d, 1);

    // ---- P2 (block 0): super-tile list offsets, units, centroids ----
    if (blockIdx.x == 0) {
        uint32_t *ucnt = reinterpret_cast<uint32_t *>(fsm);  // [nsk] units per key
        const unsigned long long Pc = block_scan(
            nsk, [&](int i) { return __ldcg(d.skey_cnt + i); },
            [&](int i, unsigned long long pre, uint32_t c) {
                d.skey_cur[i] = (uint32_t)pre;
                d.skey_start[i] = (uint32_t)pre;
                ucnt[i] = (c + UNIT_G - 1) / UNIT_G;
            },
            s_warp);
        const bool skip = Pc > d.capC;
        if (tid == 0) {
            d.stats[0] = d.stats[1] = d.stats[2] = 0ull;
            d.stats[5] = Pc;
            d.stats[6] = skip ? 0ull : Pc;
            if (skip) {
                record_status(d.status, DGSM_ERR_WORKSPACE);
                d.ctl->skip = 1u;
            }
        }
        const unsigned long long nu = block_scan(
            nsk, [&](int i) { return ucnt[i]; },
            [&](int i, unsigned long long pre, uint32_t) { d.unit_off[i] = (uint32_t)pre; }, s_warp);
        if (tid == 0) {
            d.ctl->n_units = skip ? 0ull : nu;
            d.stats[7] = skip ? 0ull : nu;
        }
        for (int o = warp; o < d.segs.n; o += FR_THREADS / 32) centroid_final_warp(d.cen_part, d.cen_bps, o, d.centroids);
    }
    if (!grid_sync(d, 2)) return;
    stamp(d, 2);

    // ---- P3: super-tile lists; the fine-binning units ----
    const unsigned long long n_units = __ldcg(&d.ctl->n_units);
    for (int64_t i = gtid; i < (int64_t)n_units; i += gstride) {
        // unit i belongs to the last key whose first unit is <= i (empty keys
        // share their offset with the next key, which the search passes over)
        int lo = 0, hi = nsk;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldcg(d.unit_off + mid) <= (uint32_t)i) lo = mid; else hi = mid;
        }
        const uint32_t s0 = __ldcg(d.skey_start + lo), e0 = s0 + __ldcg(d.skey_cnt + lo);
        const uint32_t U = (e0 - s0 + UNIT_G - 1) / UNIT_G, u0 = __ldcg(d.unit_off + lo), j = (uint32_t)i - u0;
        Unit u;
        u.key = (uint32_t)lo;
        u.start = s0 + j * UNIT_G;
        u.end = min(s0 + (j + 1) * UNIT_G, e0);
        u.ju = j | (U << 16);
        u.u0 = u0;
        u.pad0 = u.pad1 = u.pad2 = 0u;
        d.units[i] = u;
    }
    if (!__ldcg(&d.ctl->skip)) {
        // each block counts its (light, Gaussian) pairs per key in shared memory,
        // reserves one range per key, then writes: a handful of global atomics
        // per key and block instead of one per warp (a few keys hold most pairs)
        uint32_t *hist = reinterpret_cast<uint32_t *>(fsm);  // [nsk]
        uint32_t *curs = hist + nsk;                          // [nsk]
        for (int k = tid; k < nsk; k += FR_THREADS) hist[k] = 0u;
        __syncthreads();
        const int64_t total = (int64_t)d.L * N;
        const float4 *scones = d.cones + 2 * d.n_tiles;
        for (int pass = 0; pass < 2; ++pass) {
            for (int64_t idx = gtid; idx < total; idx += gstride) {
                const int l = (int)(idx / N);
                const uint32_t g = (uint32_t)(idx - (int64_t)l * N);
                uint32_t *cnt = pass == 0 ? hist : curs;
                auto take = [&](int sidx) {
                    const uint32_t pos = atomicAdd(&cnt[l * d.n_super + sidx], 1u);
                    if (pass == 1 && pos < d.capC) d.cvals[pos] = g;
                };
                if (d.n_super <= 64) {
                    for (unsigned long long sm = __ldcg(d.smask + idx); sm; sm &= sm - 1) take(__ffsll(sm) - 1);
                } else {
                    const BinRec br = frame_binrec(d, s_pose, l, g);
                    const int mode = (int)br.b.y;
                    if (mode != 0)
                        for (int sidx = 0; sidx < d.n_super; ++sidx)
                            if (mode == 2 || cone_overlap(br, scones + 2 * sidx)) take(sidx);
                }
            }
            __syncthreads();
            if (pass == 0) {
                for (int k = tid; k < nsk; k += FR_THREADS) {
                    const uint32_t c = hist[k];
                    curs[k] = c ? atomicAdd(d.skey_cur + k, c) : 0u;
                }
                __syncthreads();
            }
        }
    }
    if (!grid_sync(d, 3)) return;
    stamp(d, 3);

    // ---- P4: fine binning of the units, per-tile counts ----
    {
        const FineSmem sm = fine_smem(fsm);
        for (int k = tid; k < FB_WARPS * 64 * 3; k += blockDim.x) (&sm.wm[0][0][0])[k] = 0u;
        for (;;) {
            if (tid == 0) s_next = atomicAdd(&d.ctl->unit_counter, 1u);
            __syncthreads();
            const unsigned long long u = s_next;
            if (u >= n_units) break;
            const Unit U = load_unit(d.units + u);
            fine_count_unit(
                U, u, d.cvals, [&](int l, uint32_t g) { return frame_binrec(d, s_pose, l, g); }, d.tx, d.ty, d.sx,
                d.n_tiles, d.n_super, d.cones, d.fmask, nullptr, sm);
            if (tid < 64) {
                const uint32_t c = sm.running[tid];
                d.fcnt[64ull * u + tid] = c;
                if (c) {
                    const int l = (int)(U.key / (uint32_t)d.n_super), sidx = (int)(U.key - (uint32_t)l * d.n_super);
                    const int a = (sidx / d.sx) * SUPER + tid / SUPER, b = (sidx % d.sx) * SUPER + tid % SUPER;
                    atomicAdd(d.tile_cnt + l * d.n_tiles + a * d.tx + b, c);
                }
            }
        }
    }
    if (!grid_sync(d, 4)) return;
    stamp(d, 4);

    // ---- P5 (block 0): tile offsets, work items ----
    if (blockIdx.x == 0) {
        const unsigned long long P = block_scan(
            ntk, [&](int i) { return __ldcg(d.tile_cnt + i); },
            [&](int i, unsigned long long pre, uint32_t c) {
                d.ts[i] = (uint32_t)pre;
                d.te[i] = (uint32_t)pre + c;
                d.tcur[i] = (uint32_t)pre;
            },
            s_warp);
        const bool over = P > d.cap;
        const bool skip = over || __ldcg(&d.ctl->skip);
        if (tid == 0) {
            d.stats[3] = P;
            d.stats[4] = skip ? 0ull : P;
            if (over) record_status(d.status, DGSM_ERR_WORKSPACE);
            d.ctl->skip = skip ? 1u : 0u;
        }
        if (skip)  // no pairs kept: every tile's list is empty (T = 1)
            for (int i = tid; i < ntk; i += FR_THREADS) d.ts[i] = d.te[i] = 0u;
        __syncthreads();
        const uint32_t item = (uint32_t)(ITEM_CHUNKS * d.chunk);
        const unsigned long long n_items = block_scan(
            ntk,
            [&](int i) {
                const uint32_t c = __ldcg(d.te + i) - __ldcg(d.ts + i);
                return c == 0u ? 1u : (c + item - 1u) / item;
            },
            [&](int i, unsigned long long pre, uint32_t) { d.item_off[i] = (uint32_t)pre; }, s_warp);
        if (tid == 0) d.ctl->n_items = n_items;
    }
    if (!grid_sync(d, 5)) return;
    stamp(d, 5);

    // ---- P6: the tiles' work items; per-tile lists from the fine bitmaps ----
    {
        const uint32_t item = (uint32_t)(ITEM_CHUNKS * d.chunk);
        for (int64_t k = gtid; k < ntk; k += gstride) {
            const uint32_t s0 = __ldcg(d.ts + k), e0 = __ldcg(d.te + k), o = __ldcg(d.item_off + k);
            const uint32_t n = e0 == s0 ? 1u : (e0 - s0 + item - 1u) / item;
            for (uint32_t q = 0; q < n; ++q) {
                Item it;
                it.key = (uint32_t)k;
                it.start = s0 + q * item;
                it.end = min(s0 + (q + 1) * item, e0);
                it.n_items = n;
                d.items[o + q] = it;
            }
        }
    }
    if (!__ldcg(&d.ctl->skip)) {
        uint32_t *gidx = reinterpret_cast<uint32_t *>(fsm);  // [UNIT_G]
        for (;;) {
            __syncthreads();  // gidx and s_next of the previous unit are no longer read
            if (tid == 0) s_next = atomicAdd(&d.ctl->emit_counter, 1u);
            __syncthreads();
            const unsigned long long u = s_next;
            if (u >= n_units) break;
            const Unit U = load_unit(d.units + u);
            const int l = (int)(U.key / (uint32_t)d.n_super), sidx = (int)(U.key - (uint32_t)l * d.n_super);
            const int sa = sidx / d.sx, sb = sidx - sa * d.sx;
            const int ng = (int)(U.end - U.start);
            for (int e = tid; e < ng; e += FR_THREADS) gidx[e] = __ldcg(d.cvals + U.start + e);
            __syncthreads();
            const uint32_t *um = d.fmask + u * (64ull * 3 * MASK_WORDS);
            for (int jj = 0; jj < 8; ++jj) {
                const int t = warp * 8 + jj;
                const int a = sa * SUPER + t / SUPER, b = sb * SUPER + t % SUPER;
                if (a >= d.ty || b >= d.tx) continue;
                const uint32_t c = d.fcnt[64ull * u + t];
                if (c == 0u) continue;
                const uint32_t key = (uint32_t)l * (uint32_t)d.n_tiles + (uint32_t)(a * d.tx + b);
                uint32_t pos0 = 0u;
                if (lane == 0) pos0 = atomicAdd(d.tcur + key, c);
                pos0 = __shfl_sync(FULLMASK, pos0, 0);
                emit_tile(um, t, ng, pos0, gidx, d.vals, nullptr, 0u, d.cap);
            }
        }
    }
    if (!grid_sync(d, 6)) return;
    stamp(d, 6);

    // ---- P7: the dynamic atlases (closed form, Eqs. 3-4) ----
    tiles_worker<float, 8>(reinterpret_cast<const float4 *>(d.brec), d.vals, d.items, &d.ctl->n_items,
                           &d.ctl->item_counter, d.radii_d, d.Kd, d.Hd, d.Wd, d.tx, d.n_tiles, N, d.chunk, d.accum,
                           d.done, d.dyn, d.stats, nullptr, nullptr, MAP_OCTA, fsm);
    if (!grid_sync(d, 7)) return;
    stamp(d, 7);

    // ---- P8: attenuation of every receiver; relight of the avatars ----
    {
        const AttTabs at = att_tabs(d, fsm);
        float4 *tab = reinterpret_cast<float4 *>(reinterpret_cast<char *>(fsm) + ATT_TAB_BYTES);  // [2 FR_TAB]
        float *shs = reinterpret_cast<float *>(tab + 2 * FR_TAB);                               // [27]
        float *cen = shs + 28;                                                                   // [3 n_obj]
        for (int k = tid; k < 27; k += FR_THREADS) shs[k] = d.sh[k];
        for (int k = tid; k < 3 * d.segs.n; k += FR_THREADS) cen[k] = __ldcg(d.centroids + k);
        __syncthreads();
        const float wd = d.wd;
        // every block relights its avatars first, then attenuates its static
        // receivers (measured: faster than mixing the two on an SM, whose
        // gathers then lose shared L1 and warps to the relight's table passes)
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                // static receivers: FR_ATT_U per thread, blockDim apart
                const int64_t span = (int64_t)FR_ATT_U * FR_THREADS;
                for (int64_t base = (int64_t)blockIdx.x * span; base < d.n_static; base += (int64_t)gridDim.x * span) {
                    float px[FR_ATT_U], py[FR_ATT_U], pz[FR_ATT_U], acc[FR_ATT_U];
#pragma unroll
                    for (int u = 0; u < FR_ATT_U; ++u) {
                        const int64_t q = base + u * FR_THREADS + tid;
                        const bool ok = q < d.n_static;
                        px[u] = ok ? __ldg(d.q_means + 3 * q) : 0.f;
                        py[u] = ok ? __ldg(d.q_means + 3 * q + 1) : 0.f;
                        pz[u] = ok ? __ldg(d.q_means + 3 * q + 2) : 0.f;
                    }
                    att_batch<FR_ATT_U>(d, at, px, py, pz, acc);
#pragma unroll
                    for (int u = 0; u < FR_ATT_U; ++u) {
                        const int64_t q = base + u * FR_THREADS + tid;
                        if (q >= d.n_static) continue;
                        const float f = 1.0f - wd + wd * acc[u];
                        __stcs(d.cout + 3 * q, d.cin[3 * q] * f);
                        __stcs(d.cout + 3 * q + 1, d.cin[3 * q + 1] * f);
                        __stcs(d.cout + 3 * q + 2, d.cin[3 * q + 2] * f);
                    }
                }
            } else {
                // avatar receivers in groups of FR_RG consecutive Gaussians, a group
                // per thread; groups are dealt warp-major across the blocks (warp 0
                // of every block, then warp 1, ...) so that few avatars fill few
                // whole warps spread over every SM, and warps without a group skip
                // the sums.  The relight table passes through shared memory FR_TAB
                // directions at a time (every block runs the same rounds).
                const int64_t n_groups = (N + FR_RG - 1) / FR_RG;
                const int64_t per_round = (int64_t)gridDim.x * FR_THREADS;
                const int rounds = (int)((n_groups + per_round - 1) / per_round);
                const int M = d.nth * d.nph;
                for (int rd = 0; rd < rounds; ++rd) {
                    const int64_t G =
                        (((int64_t)rd * (FR_THREADS / 32) + warp) * gridDim.x + blockIdx.x) * 32 + lane;
                    const bool busy = __any_sync(FULLMASK, G < n_groups);
                    float3 n[FR_RG];
#pragma unroll
                    for (int r = 0; r < FR_RG; ++r) {
                        const int64_t g = G * FR_RG + r;
                        n[r] = make_float3(0.f, 0.f, 1.f);  // a padding slot: summed, never written
                        if (G < n_groups && g < N) {
                            const int o = d.segs.n == 1 ? 0 : seg_find(d.segs, g);
                            const float *pr = s_pose[o];
                            const float3 m =
                                pose_point(pr, d.rest_means[3 * g], d.rest_means[3 * g + 1], d.rest_means[3 * g + 2]);
                            const float4 q = pose_quat(pr, reinterpret_cast<const float4 *>(d.rest_quats)[g]);
                            n[r] = relight_axis_normal_v(m.x, m.y, m.z, q.x, q.y, q.z, q.w, d.scales[3 * g],
                                                         d.scales[3 * g + 1], d.scales[3 * g + 2], cen[3 * o],
                                                         cen[3 * o + 1], cen[3 * o + 2]);
                        }
                    }
                    float4 acc[FR_RG];
#pragma unroll
                    for (int r = 0; r < FR_RG; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int j0 = 0; j0 < M; j0 += FR_TAB) {
                        const int j1 = min(j0 + FR_TAB, M);
                        __syncthreads();  // the previous piece of the table is no longer read
                        relight_table_fill(shs, j0, j1, d.nth, d.nph, tab);
                        __syncthreads();
                        if (busy) relight_accumulate_add<FR_RG>(tab, j1 - j0, d.rq, n, acc);
                    }
#pragma unroll
                    for (int r = 0; r < FR_RG; ++r) {
                        const int64_t g = G * FR_RG + r;
                        if (G >= n_groups || g >= N) continue;
                        const float *pr = s_pose[d.segs.n == 1 ? 0 : seg_find(d.segs, g)];
                        const float3 m =
                            pose_point(pr, d.rest_means[3 * g], d.rest_means[3 * g + 1], d.rest_means[3 * g + 2]);
                        float px1[1] = {m.x}, py1[1] = {m.y}, pz1[1] = {m.z}, ta[1];
                        att_batch<1>(d, at, px1, py1, pz1, ta);
                        const float f = 1.0f - wd + wd * ta[0];
                        const int64_t q = d.n_static + g;
                        relight_write_rgb(acc[r], d.reps, d.rt_max, d.rgamma, d.cin[3 * q] * f, d.cin[3 * q + 1] * f,
                                          d.cin[3 * q + 2] * f, d.cout, q);
                    }
                }
            }
        }
    }
    if (d.phase_ns) {
        __syncthreads();
        if (tid == 0 && atomicAdd(&d.ctl->done_blocks, 1u) == gridDim.x - 1) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            d.phase_ns[8] = t;
        }
    }
}


}  // namespace
}  // namespace dgsm

namespace dgsm {
namespace {

__global__ void frame_cones_kernel(int H, int W, int tx, int ty, int sx, int sy, float4 *__restrict__ cones) {
    rect_cones_one(blockIdx.x * blockDim.x + threadIdx.x, H, W, 8, tx, ty, sx, sy, cones, MAP_OCTA);
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_frame(dgsm_ctx *ctx, const dgsm_crowd_frame_args *a, const dgsm_params &p,
                const dgsm_relight_params &rp) {
    auto bad = [&](const char *m) { return fail(ctx, DGSM_ERR_INVALID_ARG, std::string("crowd_frame: ") + m); };
    if (p.tile != 8) return bad("tile must be 8");
    if (p.atlas_dtype != DGSM_F32) return bad("atlas_dtype must be DGSM_F32");
    if (p.atlas_map != MAP_OCTA) return bad("the octahedral map only (atlas_map 0)");
    if (p.chunk < 16 || p.chunk > 192) return bad("chunk must be in 16..192");
    if (!(p.kappa >= 0.f) || !(p.eps_cull > 0.f)) return bad("kappa >= 0 and eps_cull > 0 required");
    if (p.beta_mode < 1 || p.beta_mode > 4) return bad("beta_mode must be 1..4");
    if (p.max_pairs < 1 || p.max_pairs >= ((int64_t)1 << 31)) return bad("max_pairs must be in 1..2^31-1");
    if (rp.n_theta < 1 || rp.n_phi < 1 || (int64_t)rp.n_theta * rp.n_phi > 6144)
        return bad("need 1 <= n_theta * n_phi <= 6144");
    if (!(rp.q > 0.0f) || !(rp.eps >= 0.0f) || !(rp.t_max >= 0.0f)) return bad("need q > 0, eps >= 0, t_max >= 0");
    if (a->L < 1 || a->L > 64 || !a->lights) return bad("need 1..64 lights");
    if (a->H < 1 || a->W < 1 || a->H > 4096 || a->W > 4096 || a->H_dyn < 1 || a->W_dyn < 1 || a->H_dyn > 4096 ||
        a->W_dyn > 4096)
        return bad("H, W, H_dyn, W_dyn must be in 1..4096");
    if (a->K < 1 || a->K > 256 || a->K_dyn < 1 || a->K_dyn > 256 || !a->radii || !a->radii_dyn)
        return bad("K, K_dyn must be in 1..256 (radii required)");
    if (a->n_static < 0 || a->n_avatar < 0 || a->n_avatar >= ((int64_t)1 << 30)) return bad("bad Gaussian counts");
    if (!a->static_atlas || !a->dyn_atlas || !a->sh || !a->centroids_out || !a->poses || !a->seg)
        return bad("null atlas, sh, centroids, poses or seg");
    if (a->n_static + a->n_avatar > 0 && (!a->q_means || !a->colors_in || !a->colors_out))
        return bad("null receiver array");
    if (a->n_avatar > 0 && (!a->rest_means || !a->rest_quats || !a->scales || !a->opac || !a->quats_out))
        return bad("null avatar array");
    if (((uintptr_t)a->rest_quats | (uintptr_t)a->quats_out) & 15) return bad("quaternion arrays must be 16-byte aligned");
    return DGSM_OK;
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_crowd_frame(dgsm_ctx *ctx, const dgsm_crowd_frame_args *a, const dgsm_params *params,
                                const dgsm_relight_params *rparams, int32_t timeout_barrier, void *stream) {
    DGSM_RANGE("dgsm_crowd_frame");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!a) return fail(ctx, DGSM_ERR_INVALID_ARG, "crowd_frame: null arguments");
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    dgsm_relight_params rp;
    if (rparams) rp = *rparams; else dgsm_default_relight_params(&rp);
    int rc = check_frame(ctx, a, p, rp);
    if (rc) return rc;
    Segs segs;
    if (!make_segs(a->seg, a->n_obj, a->n_avatar, &segs))
        return fail(ctx, DGSM_ERR_INVALID_ARG,
                    "crowd_frame: need 1 <= n_obj <= 64 and 0 = seg[0] <= ... <= seg[n_obj] = n_avatar");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;

    // geometry of the dynamic atlases (tile 8)
    const int L = a->L, Hd = a->H_dyn, Wd = a->W_dyn, Kd = a->K_dyn;
    const int tx = (Wd + 7) / 8, ty = (Hd + 7) / 8, sx = (tx + SUPER - 1) / SUPER, sy = (ty + SUPER - 1) / SUPER;
    const int n_tiles = tx * ty, n_super = sx * sy;
    const int64_t nsk = (int64_t)L * n_super, ntk = (int64_t)L * n_tiles;
    if (nsk > FR_MAX_SKEYS || ntk > FR_MAX_TKEYS)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "crowd_frame: need L x super-tiles <= 4096 and L x tiles <= 65536");
    const int64_t N = a->n_avatar, LN = (int64_t)L * N;
    const uint32_t cap = (uint32_t)p.max_pairs, capC = cap;
    const uint32_t item = (uint32_t)(ITEM_CHUNKS * p.chunk);
    const int64_t max_units = capC / UNIT_G + nsk + 1, max_items = ntk + cap / item + 1;
    int64_t longest = 0;
    for (int o = 0; o < a->n_obj; ++o) longest = std::max<int64_t>(longest, a->seg[o + 1] - a->seg[o]);
    const int bps = (int)std::max<int64_t>(
        1, std::min<int64_t>((longest + CEN_THREADS - 1) / CEN_THREADS,
                             std::max<int64_t>(1, 2 * (int64_t)ctx->num_sms / a->n_obj)));

    // workspace: the region zeroed before every launch first
    const size_t sz_ctl = al256(sizeof(FrameCtl)), sz_skc = al256(4 * (size_t)nsk), sz_tc = al256(4 * (size_t)ntk);
    const size_t sz_zero = sz_ctl + sz_skc + sz_tc;
    const size_t sizes[] = {al256(4 * (size_t)nsk),                                  // skey_cur
                            al256(4 * (size_t)nsk), al256(4 * (size_t)nsk),          // skey_start, unit_off
                            al256(4 * (size_t)ntk), al256(4 * (size_t)ntk),          // ts, te
                            al256(4 * (size_t)ntk), al256(4 * (size_t)ntk),          // tcur, item_off
                            al256(4 * (size_t)capC),                                 // cvals
                            al256(sizeof(Unit) * (size_t)max_units),                 // units
                            al256(4 * 64 * (size_t)max_units),                       // fcnt
                            al256(4 * 64 * 3 * (size_t)MASK_WORDS * max_units),      // fmask
                            al256(sizeof(Item) * (size_t)max_items),                 // items
                            al256(4 * (size_t)cap),                                  // vals
                            al256(sizeof(BuildRec) * (size_t)std::max<int64_t>(LN, 1)),  // brec
                            al256(sizeof(unsigned long long) * (size_t)std::max<int64_t>(LN, 1)),  // smask
                            al256(sizeof(double) * 4 * (size_t)bps * a->n_obj),      // cen_part
                            al256(sizeof(float) * 8 * MAX_OBJECTS)};                 // poses
    size_t total = sz_zero;
    for (size_t z : sizes) total += z;
    void *base;
    if ((rc = ws_reserve(ctx, WS_PFRAME, total, &base))) return rc;
    char *c = (char *)base;
    auto take = [&](size_t bytes) { char *r = c; c += bytes; return (void *)r; };
    FrameDev d;
    d.ctl = (FrameCtl *)take(sz_ctl);
    d.skey_cnt = (uint32_t *)take(sz_skc);
    d.tile_cnt = (uint32_t *)take(sz_tc);
    int si = 0;
    d.skey_cur = (uint32_t *)take(sizes[si++]);
    d.skey_start = (uint32_t *)take(sizes[si++]);
    d.unit_off = (uint32_t *)take(sizes[si++]);
    d.ts = (uint32_t *)take(sizes[si++]);
    d.te = (uint32_t *)take(sizes[si++]);
    d.tcur = (uint32_t *)take(sizes[si++]);
    d.item_off = (uint32_t *)take(sizes[si++]);
    d.cvals = (uint32_t *)take(sizes[si++]);
    d.units = (Unit *)take(sizes[si++]);
    d.fcnt = (uint32_t *)take(sizes[si++]);
    d.fmask = (uint32_t *)take(sizes[si++]);
    d.items = (Item *)take(sizes[si++]);
    d.vals = (uint32_t *)take(sizes[si++]);
    d.brec = (BuildRec *)take(sizes[si++]);
    d.smask = (unsigned long long *)take(sizes[si++]);
    d.cen_part = (double *)take(sizes[si++]);
    float *d_poses = (float *)take(sizes[si++]);
    // per-voxel accumulators and per-tile counters, shared with dgsm_build:
    // every user leaves them at zero, so they are cleared only when new
    const size_t acc_bytes = sizeof(float) * (size_t)L * Kd * Hd * Wd;
    const bool acc_new = ctx->ws_cap[WS_ACCUM] < acc_bytes;
    void *w_acc, *w_done;
    if ((rc = ws_reserve(ctx, WS_ACCUM, acc_bytes, &w_acc))) return rc;
    const bool done_new = ctx->ws_cap[WS_DONE] < sizeof(uint32_t) * (size_t)ntk;
    if ((rc = ws_reserve(ctx, WS_DONE, sizeof(uint32_t) * (size_t)ntk, &w_done))) return rc;
    // the tile cones depend only on the atlas size: computed when it changes
    const size_t cone_f4 = 2 * (size_t)(n_tiles + n_super) + PLANE_F4 * (size_t)n_tiles + 2 * (size_t)n_super;
    void *w_cones;
    if ((rc = ws_reserve(ctx, WS_PF_CONES, sizeof(float4) * cone_f4, &w_cones))) return rc;
    e = cudaSuccess;
    if (acc_new) e = cudaMemsetAsync(w_acc, 0, ctx->ws_cap[WS_ACCUM], s);
    if (e == cudaSuccess && done_new) e = cudaMemsetAsync(w_done, 0, ctx->ws_cap[WS_DONE], s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame: accumulator memset");
    if (ctx->pf_cones != w_cones || ctx->pf_cones_h != Hd || ctx->pf_cones_w != Wd) {
        const int nc = n_tiles + n_super;
        frame_cones_kernel<<<(nc + 127) / 128, 128, 0, s>>>(Hd, Wd, tx, ty, sx, sy, (float4 *)w_cones);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame: cones kernel");
        ctx->pf_cones = w_cones;
        ctx->pf_cones_h = Hd;
        ctx->pf_cones_w = Wd;
    }
    e = cudaMemcpyAsync(d_poses, a->poses, sizeof(float) * 8 * (size_t)a->n_obj, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, sz_zero, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame: pose copy / control memset");

    d.q_means = a->q_means;
    d.cin = a->colors_in;
    d.cout = a->colors_out;
    d.n_static = a->n_static;
    d.sat = a->static_atlas;
    d.H = a->H; d.W = a->W; d.K = a->K;
    d.radii = a->radii;
    d.rest_means = a->rest_means; d.rest_quats = a->rest_quats; d.scales = a->scales; d.opac = a->opac;
    d.av_means = const_cast<float *>(a->q_means) + 3 * a->n_static;
    d.av_quats = a->quats_out;
    d.N = N;
    d.poses = d_poses;
    d.dyn = a->dyn_atlas;
    d.Hd = Hd; d.Wd = Wd; d.Kd = Kd;
    d.radii_d = a->radii_dyn;
    d.tx = tx; d.ty = ty; d.sx = sx; d.n_tiles = n_tiles; d.n_super = n_super;
    d.lights = a->lights;
    d.L = L;
    d.kappa = p.kappa; d.eps_cull = p.eps_cull; d.wd = a->direct_frac;
    d.beta_mode = p.beta_mode == 4 ? 3 : p.beta_mode;
    d.chunk = p.chunk;
    d.sh = a->sh;
    d.rq = rp.q; d.rgamma = rp.gamma; d.rt_max = rp.t_max; d.reps = rp.eps;
    d.nth = rp.n_theta; d.nph = rp.n_phi;
    d.centroids = a->centroids_out;
    d.cen_bps = bps;
    d.cones = (const float4 *)w_cones;
    d.accum = (float *)w_acc;
    d.done = (unsigned *)w_done;
    d.status = ctx->d_status;
    d.stats = ctx->d_stats;
    d.capC = capC; d.cap = cap;
    d.max_units = (uint32_t)max_units; d.max_items = (uint32_t)max_items;
    d.timeout_barrier = timeout_barrier;
    d.segs = segs;
    d.phase_ns = nullptr;
    if (ctx->prof) {
        void *ph;
        if ((rc = ws_reserve(ctx, WS_PF_PHASE, 9 * sizeof(unsigned long long), &ph))) return rc;
        d.phase_ns = (unsigned long long *)ph;
    }

    const size_t smem = std::max({build_smem_bytes(Kd, 8, p.chunk), FINE_SMEM_BYTES, 2 * sizeof(uint32_t) * (size_t)nsk,
                                  sizeof(uint32_t) * (size_t)UNIT_G, relight_smem_bytes()});
    e = cudaFuncSetAttribute(crowd_frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame: smem attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crowd_frame_kernel, FR_THREADS, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame: occupancy query");
    if (per_sm < 1) return fail(ctx, DGSM_ERR_INVALID_ARG, "crowd_frame: the kernel does not fit an SM");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(per_sm * ctx->num_sms));
    cfg.blockDim = dim3(FR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, crowd_frame_kernel, d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame_kernel (cooperative launch)");
    return DGSM_OK;
}

// Phase times of the last frame run while the context profiled: ms_out[k] =
// time from barrier k to barrier k + 1 (k = 0: from the kernel's start; k =
// 7: to the last block's end), as block 0 saw the barriers.  Blocks.
extern "C" int dgsm_crowd_frame_phases(dgsm_ctx *ctx, double *ms_out) {
    if (!ctx || !ms_out) return DGSM_ERR_INVALID_ARG;
    if (!ctx->ws[WS_PF_PHASE]) return fail(ctx, DGSM_ERR_INVALID_ARG, "crowd_frame_phases: no profiled frame");
    cudaError_t e = cudaSetDevice(ctx->device);
    unsigned long long t[9];
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(t, ctx->ws[WS_PF_PHASE], sizeof(t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crowd_frame_phases");
    for (int k = 0; k < 8; ++k) ms_out[k] = (double)(long long)(t[k + 1] - t[k]) * 1e-6;
    return DGSM_OK;
}
