// build.cu -- Deep Gaussian Shadow Map build on sm_103a (Sec. 3.2).
//
// Pipeline per call (all on the caller's stream):
//   rect_cones_kernel   direction cones of every atlas tile and super-tile
//   prep_kernel         per (light, Gaussian): whitening matrix M = S^-1 R^T,
//                       w' = M (mu - o), beta (Eq. 5), culling radius, shell
//                       window, bounding cone
//   bin_kernel<false>   tiles overlapped by each Gaussian's cone (one warp per
//                       Gaussian, 32 cone tests at a time)
//   scan                exclusive prefix sum -> pair offsets   (one host sync)
//   bin_kernel<true>    (key = light*tiles + tile, value = Gaussian) pairs
//   radix sort          stable, by key -> per-tile lists in Gaussian order
//   tile_ranges_kernel  [start, end) of every key
//   item kernels        cut every tile's list into work items of <= ITEM
//                       Gaussians
//   build_items_kernel  persistent: blocks pull items from an atomic counter;
//                       stage the item's records with cp.async (double
//                       buffered); every (texel ray, Gaussian) pair gets the
//                       exact culling test in the Gaussian's whitened frame;
//                       the hits are compacted per warp and evaluated densely
//                       (Eq. 3 at the shells on the ray's chord through the
//                       culling ellipsoid, accumulated as per-shell increments);
//                       the last item of a tile takes the shell-wise prefix
//                       sum and T = exp(-tau) (Eq. 4).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>

#include "dgsm_internal.cuh"

#include "build_device.cuh"

namespace dgsm {
namespace {

__global__ void rect_cones_kernel(int H, int W, int tile, int tx, int ty, int sx, int sy,
                                  float4 *__restrict__ cones, int map) {
    rect_cones_one(blockIdx.x * blockDim.x + threadIdx.x, H, W, tile, tx, ty, sx, sy, cones, map);
}

__global__ void __launch_bounds__(256) prep_kernel(
    const float *__restrict__ means, const float *__restrict__ scales,
    const float *__restrict__ quats, const float *__restrict__ opac, int64_t N,
    const float *__restrict__ lights, int L, const float *__restrict__ radii, int K, float kappa,
    float eps, BuildRec *__restrict__ brec, BinRec *__restrict__ bin, int *__restrict__ status,
    const int *__restrict__ roi_k, int beta_mode) {
    // brec == nullptr: binning only (no build record)
    // roi_k (or nullptr): per light the shell range [kmin, kmax] of a region
    // of interest; Gaussians wholly beyond shell kmax cannot change it
    const int64_t total = (int64_t)L * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx / N);
        const int64_t g = idx - (int64_t)l * N;
        BinRec br;
        prep_one(idx, l, g, means, scales, quats, opac, lights, radii, K, kappa, eps, brec, br, status, roi_k,
                 beta_mode);
        bin[idx] = br;
    }
}

template <bool EMIT, bool TWO>
__global__ void __launch_bounds__(256) coarse_bin_kernel(
    const BinRec *__restrict__ bin, int64_t N, int L, int n_super, const float4 *__restrict__ scones,
    const float4 *__restrict__ scones2, uint32_t *__restrict__ counts, const uint32_t *__restrict__ offsets, uint32_t *__restrict__ ckeys,
    uint32_t *__restrict__ cvals, const unsigned long long *__restrict__ keep, uint32_t cap,
    const uint8_t *__restrict__ sact) {
    // sact (or nullptr): per (light, super-tile) 1 if it holds a texel of the
    // region of interest
    if (EMIT && *keep == 0) return;
    const int64_t total = (int64_t)L * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const float4 ga = bin[idx].a, gb = bin[idx].b;
        BinRec g;
        g.a = ga;
        g.b = gb;
        const int mode = (int)gb.y;
        const int l = (int)(idx / N);
        const uint32_t gi = (uint32_t)(idx - (int64_t)l * N);
        uint32_t c = 0, off = EMIT ? offsets[idx] : 0u;
        if (mode != 0) {
            for (int sidx = 0; sidx < n_super; ++sidx) {
                if ((!sact || sact[l * n_super + sidx]) &&
                    (mode == 2 || (TWO ? super_overlap(g, scones, scones2, sidx) : cone_overlap(g, scones + 2 * sidx)))) {
                    if (EMIT && off + c < cap) {
                        ckeys[off + c] = (uint32_t)(l * n_super + sidx);
                        cvals[off + c] = gi;
                    }
                    ++c;
                }
            }
        }
        if (!EMIT) counts[idx] = c;
    }
}

// The build's super-tile lists without a sort (dgsm_bin keeps the sorted
// lists above, whose order its output reports).  Count: each (light,
// Gaussian) keeps the mask of the super-tiles it reaches (n_super <= 64) and
// each block adds its counts per (light, super-tile) key from a shared
// histogram.  Emit: each block counts its pairs per key again from the masks,
// reserves one range per key from the key cursors, and writes its Gaussians
// there, so that a key's list is contiguous (its order follows the blocks).
template <bool TWO>
__global__ void __launch_bounds__(256) coarse_mask_kernel(
    const BinRec *__restrict__ bin, int64_t N, int L, int n_super, const float4 *__restrict__ scones,
    const float4 *__restrict__ scones2, unsigned long long *__restrict__ masks, uint32_t *__restrict__ kcnt,
    const uint8_t *__restrict__ sact) {
    extern __shared__ uint32_t hist[];  // [L n_super]
    const int nk = L * n_super;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const int64_t total = (int64_t)L * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        BinRec g;
        g.a = bin[idx].a;
        g.b = bin[idx].b;
        const int mode = (int)g.b.y;
        const int l = (int)(idx / N);
        unsigned long long m = 0ull;
        if (mode != 0)
            for (int sidx = 0; sidx < n_super; ++sidx)
                if ((!sact || sact[l * n_super + sidx]) &&
                    (mode == 2 || (TWO ? super_overlap(g, scones, scones2, sidx) : cone_overlap(g, scones + 2 * sidx))))
                    m |= 1ull << sidx;
        masks[idx] = m;
        for (unsigned long long mm = m; mm; mm &= mm - 1) atomicAdd(&hist[l * n_super + __ffsll(mm) - 1], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x)
        if (hist[k]) atomicAdd(kcnt + k, hist[k]);
}

// Key ranges from the scanned counts: [cs, ce) and the emit cursor, or
// every list empty when the pairs do not fit (keep = 0).
__global__ void key_ranges_kernel(const uint32_t *__restrict__ kcnt, int nk, const unsigned long long *__restrict__ keep,
                                  uint32_t *__restrict__ cs, uint32_t *__restrict__ ce, uint32_t *__restrict__ cur) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const bool kept = *keep != 0;
    const uint32_t s0 = kept ? cs[k] : 0u;
    cs[k] = s0;
    ce[k] = kept ? s0 + kcnt[k] : 0u;
    cur[k] = s0;
}

__global__ void __launch_bounds__(256) coarse_scatter_kernel(
    const unsigned long long *__restrict__ masks, int64_t N, int L, int n_super, uint32_t *__restrict__ cur,
    uint32_t *__restrict__ cvals, const unsigned long long *__restrict__ keep, uint32_t cap) {
    if (*keep == 0) return;
    extern __shared__ uint32_t sh[];  // [2][L n_super]: counts, then this block's cursors
    const int nk = L * n_super;
    uint32_t *hist = sh, *bcur = sh + nk;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const int64_t total = (int64_t)L * N;
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t *cnt = pass == 0 ? hist : bcur;
        for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
             idx += (int64_t)gridDim.x * blockDim.x) {
            const int l = (int)(idx / N);
            const uint32_t gi = (uint32_t)(idx - (int64_t)l * N);
            for (unsigned long long m = masks[idx]; m; m &= m - 1) {
                const uint32_t pos = atomicAdd(&cnt[l * n_super + __ffsll(m) - 1], 1u);
                if (pass == 1 && pos < cap) cvals[pos] = gi;
            }
        }
        __syncthreads();
        if (pass == 0) {
            for (int k = threadIdx.x; k < nk; k += blockDim.x) bcur[k] = hist[k] ? atomicAdd(cur + k, hist[k]) : 0u;
            __syncthreads();
        }
    }
}

// Work units of pass B: unit_cnt[key] = ceil(list length / UNIT_G).
__global__ void unit_count_kernel(const uint32_t *__restrict__ cs, const uint32_t *__restrict__ ce,
                                  int n_keys, uint32_t *__restrict__ unit_cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_keys) unit_cnt[k] = (ce[k] - cs[k] + UNIT_G - 1) / UNIT_G;
}


__global__ void unit_fill_kernel(const uint32_t *__restrict__ cs, const uint32_t *__restrict__ ce,
                                 int n_keys, const uint32_t *__restrict__ unit_off,
                                 Unit *__restrict__ units) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_keys) return;
    const uint32_t s0 = cs[k], e0 = ce[k];
    const uint32_t U = (e0 - s0 + UNIT_G - 1) / UNIT_G, u0 = unit_off[k];
    for (uint32_t j = 0; j < U; ++j) {
        Unit u;
        u.key = (uint32_t)k;
        u.start = s0 + j * UNIT_G;
        u.end = min(s0 + (j + 1) * UNIT_G, e0);
        u.ju = j | (U << 16);
        u.u0 = u0;
        u.pad0 = u.pad1 = u.pad2 = 0u;
        units[u0 + j] = u;
    }
}

__global__ void __launch_bounds__(256, 5) fine_count_kernel(
    const Unit *__restrict__ units, const unsigned long long *__restrict__ n_units_dev,
    const uint32_t *__restrict__ cvals, const BinRec *__restrict__ bin, int64_t N, int tx, int ty,
    int sx, int n_tiles, int n_super, const float4 *__restrict__ cones, uint32_t *__restrict__ fcnt,
    uint32_t *__restrict__ fmask, const uint8_t *__restrict__ tact) {
    __shared__ __align__(16) char smem[FINE_SMEM_BYTES];
    const FineSmem sm = fine_smem(smem);
    const unsigned long long n_units = *n_units_dev;
    const int tid = threadIdx.x;
    for (int k = tid; k < FB_WARPS * 64 * 3; k += blockDim.x) (&sm.wm[0][0][0])[k] = 0u;
    for (unsigned long long u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit U = units[u];
        fine_count_unit(
            U, u, cvals, [&](int l, uint32_t g) { return bin[(int64_t)l * N + g]; }, tx, ty, sx, n_tiles, n_super,
            cones, fmask, tact, sm);
        const uint32_t j = U.ju & 0xffffu, nU = U.ju >> 16;
        if (tid < 64) fcnt[64u * U.u0 + (uint32_t)tid * nU + j] = sm.running[tid];
    }
}

// Pass B, emit: expand the count pass's bitmaps into pairs at the scanned
// offsets (no tests).  A warp owns 8 tiles; lane = Gaussian within a word.
__global__ void __launch_bounds__(256) fine_emit_kernel(
    const Unit *__restrict__ units, const unsigned long long *__restrict__ n_units_dev,
    const uint32_t *__restrict__ cvals, int tx, int ty, int sx, int n_tiles, int n_super,
    const uint32_t *__restrict__ fmask, const uint32_t *__restrict__ foff, uint32_t *__restrict__ vals,
    uint32_t *__restrict__ keys, const unsigned long long *__restrict__ keep, uint32_t cap) {
    if (*keep == 0) return;
    __shared__ uint32_t gidx[UNIT_G];
    const unsigned long long n_units = *n_units_dev;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (unsigned long long u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit U = units[u];
        const int l = (int)(U.key / (uint32_t)n_super), sidx = (int)(U.key - (uint32_t)l * n_super);
        const int sa = sidx / sx, sb = sidx - sa * sx;
        const uint32_t j = U.ju & 0xffffu, nU = U.ju >> 16;
        const int ng = (int)(U.end - U.start);
        __syncthreads();
        for (int e = tid; e < ng; e += blockDim.x) gidx[e] = cvals[U.start + e];
        __syncthreads();
        const uint32_t *um = fmask + (size_t)u * 64 * 3 * MASK_WORDS;
        for (int jj = 0; jj < 8; ++jj) {
            const int t = warp * 8 + jj;
            const int a = sa * SUPER + t / SUPER, b = sb * SUPER + t % SUPER;
            if (a >= ty || b >= tx) continue;
            const uint32_t pos0 = foff[64u * U.u0 + (uint32_t)t * nU + j];
            const uint32_t key = (uint32_t)l * (uint32_t)n_tiles + (uint32_t)(a * tx + b);
            emit_tile(um, t, ng, pos0, gidx, vals, keys, key, cap);
        }
    }
}

// Tile ranges of the two-level layout: the pairs of tile t of super key k
// run from its unit-0 entry to the end of its last unit's entry.
__global__ void fine_ranges_kernel(const Unit *__restrict__ units,
                                   const unsigned long long *__restrict__ n_units_dev,
                                   const uint32_t *__restrict__ fcnt, const uint32_t *__restrict__ foff,
                                   const unsigned long long *__restrict__ keep, int n_super, int sx,
                                   int tx, int ty, int n_tiles, uint32_t *__restrict__ ts,
                                   uint32_t *__restrict__ te) {
    if (*keep == 0) return;  // no pairs kept: every tile stays empty
    const unsigned long long n_units = *n_units_dev;
    const unsigned long long total = n_units * 64ull;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long u = e >> 6;
        const Unit U = units[u];
        const uint32_t j = U.ju & 0xffffu, nU = U.ju >> 16;
        if (j != 0) continue;
        const int t = (int)(e & 63);
        const int l = (int)(U.key / (uint32_t)n_super), sidx = (int)(U.key - (uint32_t)l * n_super);
        const int a = (sidx / sx) * SUPER + t / SUPER, b = (sidx % sx) * SUPER + t % SUPER;
        if (a >= ty || b >= tx) continue;
        const uint32_t first = 64u * U.u0 + (uint32_t)t * nU;
        const uint32_t key = (uint32_t)l * (uint32_t)n_tiles + (uint32_t)(a * tx + b);
        ts[key] = foff[first];
        te[key] = foff[first + nU - 1] + fcnt[first + nU - 1];
    }
}

// The pairs the build keeps: all of them, or none (status DGSM_ERR_WORKSPACE)
// when they do not fit the buffers sized for `cap`.
__global__ void keep_pairs_kernel(const unsigned long long *__restrict__ total,
                                  unsigned long long cap, unsigned long long *__restrict__ keep,
                                  int *__restrict__ status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long P = *total;
    if (P > cap) {
        *keep = 0;
        record_status(status, DGSM_ERR_WORKSPACE);
    } else {
        *keep = P;
    }
}

__global__ void tile_ranges_kernel(const uint32_t *__restrict__ keys,
                                   const unsigned long long *__restrict__ d_P, uint32_t nkeys,
                                   uint32_t *__restrict__ start, uint32_t *__restrict__ end) {
    const int64_t P = (int64_t)*d_P;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[p];
        if (k >= nkeys) continue;
        if (p == 0 || keys[p - 1] != k) start[k] = (uint32_t)p;
        if (p == P - 1 || keys[p + 1] != k) end[k] = (uint32_t)(p + 1);
    }
}

// Items per key: ceil(count / item) (one, possibly empty, for an empty tile).
__global__ void item_count_kernel(const uint32_t *__restrict__ ts, const uint32_t *__restrict__ te,
                                  int nkeys, uint32_t item, uint32_t *__restrict__ n_items) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    const uint32_t c = te[k] - ts[k];
    n_items[k] = c == 0 ? 1u : (c + item - 1) / item;
}

__global__ void item_expand_kernel(const uint32_t *__restrict__ ts, const uint32_t *__restrict__ te,
                                   int nkeys, uint32_t item, const uint32_t *__restrict__ item_off,
                                   Item *__restrict__ items) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    const uint32_t s = ts[k], e = te[k];
    const uint32_t n = e == s ? 1u : (e - s + item - 1) / item;
    const uint32_t o = item_off[k];
    for (uint32_t q = 0; q < n; ++q) {
        Item it;
        it.key = (uint32_t)k;
        it.start = s + q * item;
        it.end = min(s + (q + 1) * item, e);
        it.n_items = n;
        items[o + q] = it;
    }
}

template <typename OutT, int T>
__global__ void __launch_bounds__(BT_THREADS, DGSM_BT_MIN_BLOCKS) build_tiles_kernel(
    const float4 *__restrict__ brec, const uint32_t *__restrict__ vals,
    const Item *__restrict__ items, const unsigned long long *__restrict__ n_items_total,
    unsigned int *__restrict__ item_counter, const float *__restrict__ radii, int K, int H, int W,
    int tx, int n_tiles, int64_t N, int chunk, float *__restrict__ accum,
    unsigned int *__restrict__ done, OutT *__restrict__ atlas,
    unsigned long long *__restrict__ stats, const uint8_t *__restrict__ roi_mask,
    const int *__restrict__ roi_k, int map) {
    extern __shared__ float4 smem4[];
    tiles_worker<OutT, T>(brec, vals, items, n_items_total, item_counter, radii, K, H, W, tx, n_tiles, N, chunk,
                          accum, done, atlas, stats, roi_mask, roi_k, map, smem4);
}

template <typename OutT, int T>
int launch_tiles(dgsm_ctx *ctx, const BuildRec *brec, const uint32_t *vals, const Item *items,
                 const unsigned long long *n_items, unsigned int *counter, const float *radii, int K,
                 int H, int W, int tx, int n_tiles, int64_t N, int chunk, float *accum, unsigned int *done,
                 void *atlas, cudaStream_t s, const uint8_t *roi_mask, const int *roi_k, int map) {
    const size_t smem = build_smem_bytes(K, T, chunk);
    cudaError_t e = cudaFuncSetAttribute(build_tiles_kernel<OutT, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: smem attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_tiles_kernel<OutT, T>, BT_THREADS, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: occupancy query");
    const int grid = std::max(1, per_sm) * ctx->num_sms;
    build_tiles_kernel<OutT, T><<<grid, BT_THREADS, smem, s>>>(
        reinterpret_cast<const float4 *>(brec), vals, items, n_items, counter, radii, K, H, W, tx,
        n_tiles, N, chunk, accum, done, (OutT *)atlas, ctx->d_stats, roi_mask, roi_k, map);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "build_tiles_kernel");
}

template <typename OutT>
int launch_build_items(dgsm_ctx *ctx, const BuildRec *brec, const uint32_t *vals, const Item *items,
                       const unsigned long long *n_items, unsigned int *counter, const float *radii,
                       int K, int H, int W, int tile, int tx, int n_tiles, int64_t N, int chunk,
                       float *accum, unsigned int *done, void *atlas, cudaStream_t s,
                       const uint8_t *roi_mask, const int *roi_k, int map) {
    if (tile == 16)
        return launch_tiles<OutT, 16>(ctx, brec, vals, items, n_items, counter, radii, K, H, W, tx, n_tiles, N,
                                      chunk, accum, done, atlas, s, roi_mask, roi_k, map);
    return launch_tiles<OutT, 8>(ctx, brec, vals, items, n_items, counter, radii, K, H, W, tx, n_tiles, N,
                                 chunk, accum, done, atlas, s, roi_mask, roi_k, map);
}
struct RoiDev {
    const uint8_t *mask = nullptr;  // [L][H][W] texels of the region
    const uint8_t *tact = nullptr;  // [L][n_tiles] tiles holding one of them
    const uint8_t *sact = nullptr;  // [L][n_super] super-tiles holding one of them
    const int *krange = nullptr;    // [L][2] shell range kmin, kmax (kmax < 0: empty)
};

struct BinOut {
    int64_t P = 0;
    uint32_t *keys = nullptr, *vals = nullptr;
    uint32_t *ts = nullptr, *te = nullptr;
    BuildRec *brec = nullptr;
    int tx = 0, ty = 0, n_tiles = 0;
};

int check_common(dgsm_ctx *ctx, const float *means, const float *scales, const float *opac,
                 int64_t n, const float *lights, int L, int H, int W, const float *radii, int K,
                 const dgsm_params &p) {
    if (n < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!means || !scales || !opac))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "null Gaussian array");
    if (n >= (int64_t)1 << 30) return fail(ctx, DGSM_ERR_INVALID_ARG, "n >= 2^30");
    if (!lights || L < 1 || L > 64) return fail(ctx, DGSM_ERR_INVALID_ARG, "need 1..64 lights");
    if (H < 1 || W < 1 || H > 4096 || W > 4096) return fail(ctx, DGSM_ERR_INVALID_ARG, "H, W must be in 1..4096");
    if (!radii || K < 1 || K > 256) return fail(ctx, DGSM_ERR_INVALID_ARG, "K must be in 1..256");
    if (p.tile != 4 && p.tile != 8 && p.tile != 16) return fail(ctx, DGSM_ERR_INVALID_ARG, "tile must be 4, 8 or 16");
    // the tile kernel's staging gives each of its 256 threads at most three of
    // a chunk's 4-float4 records: at most 3 x 256 / 4 = 192 records
    if (p.chunk < 16 || p.chunk > 192) return fail(ctx, DGSM_ERR_INVALID_ARG, "chunk must be in 16..192");
    if (!(p.kappa >= 0.f) || !(p.eps_cull > 0.f)) return fail(ctx, DGSM_ERR_INVALID_ARG, "kappa >= 0 and eps_cull > 0 required");
    if (p.beta_mode < 1 || p.beta_mode > 4) return fail(ctx, DGSM_ERR_INVALID_ARG, "beta_mode must be 1..4");
    if (p.atlas_map != MAP_OCTA && p.atlas_map != MAP_CUBE) return fail(ctx, DGSM_ERR_INVALID_ARG, "atlas_map must be 0 or 1");
    if (p.atlas_map == MAP_CUBE && (H != 6 * W || W % p.tile != 0 || W > 4096))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "cube atlas: H = 6 F, F a multiple of the tile, F <= 4096");
    return DGSM_OK;
}

static int key_bits(int64_t n_keys) {
    int bits = 0;
    while (bits < 32 && ((uint64_t)(n_keys - 1) >> bits) != 0) ++bits;
    return bits;
}

// Reads a device counter (and the status word) with one blocking copy.
static int read_count(dgsm_ctx *ctx, const unsigned long long *d, cudaStream_t s,
                      unsigned long long *out) {
    cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned + 1, ctx->d_status, sizeof(int),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: pair count");
    const int st = *(int *)(ctx->h_pinned + 1);
    if (st != DGSM_OK) {
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
        return fail(ctx, st, "a Gaussian has a non-finite field or a non-positive scale");
    }
    *out = ctx->h_pinned[0];
    return DGSM_OK;
}

// prep + two-level binning + tile ranges.  With max_pairs = 0 it blocks
// twice (after each level's count) to size the pair buffers exactly; with
// max_pairs > 0 both levels' buffers hold max_pairs pairs and the counts stay
// on the device.  want_keys: also write each pair's key (dgsm_bin).
int run_binning(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                const float *opac, int64_t N, const float *lights, int L, int H, int W,
                const float *radii, int K, const dgsm_params &p, bool build_records, bool want_keys,
                cudaStream_t s, BinOut *out, const RoiDev *roi = nullptr) {
    const int tile = p.tile;
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    const int sx = (tx + SUPER - 1) / SUPER, sy = (ty + SUPER - 1) / SUPER;
    const int n_tiles = tx * ty, n_super = sx * sy;
    out->tx = tx; out->ty = ty; out->n_tiles = n_tiles;
    const int64_t LN = (int64_t)L * N;
    const int64_t nkeys = (int64_t)L * n_tiles, nskeys = (int64_t)L * n_super;
    void *w_br, *w_bin, *w_cnt, *w_cones, *w_rng, *w_crng;
    int rc;
    if ((rc = ws_reserve(ctx, WS_BUILD_REC, build_records ? sizeof(BuildRec) * (size_t)LN : 256, &w_br)))
        return rc;
    if ((rc = ws_reserve(ctx, WS_BIN_REC, sizeof(BinRec) * (size_t)LN, &w_bin))) return rc;
    if ((rc = ws_reserve(ctx, WS_COUNTS, sizeof(uint32_t) * (size_t)LN, &w_cnt))) return rc;
    if ((rc = ws_reserve(ctx, WS_CONES,
                         sizeof(float4) * (size_t)(2 * (n_tiles + n_super) + PLANE_F4 * n_tiles + 2 * n_super),
                         &w_cones)))
        return rc;
    if ((rc = ws_reserve(ctx, WS_RANGES, 2 * sizeof(uint32_t) * (size_t)nkeys, &w_rng))) return rc;
    if ((rc = ws_reserve(ctx, WS_CRANGES, 2 * sizeof(uint32_t) * (size_t)nskeys, &w_crng))) return rc;
    out->brec = (BuildRec *)w_br;
    out->ts = (uint32_t *)w_rng;
    out->te = out->ts + nkeys;
    uint32_t *cs = (uint32_t *)w_crng, *ce = cs + nskeys;
    cudaError_t e = cudaMemsetAsync(w_rng, 0, 2 * sizeof(uint32_t) * (size_t)nkeys, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w_crng, 0, 2 * sizeof(uint32_t) * (size_t)nskeys, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_stats, 0, 8 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: memset");
    out->P = 0;
    if (N == 0) return DGSM_OK;
    unsigned long long *d_pairs = ctx->d_stats + 3, *d_keep = ctx->d_stats + 4;
    unsigned long long *d_cpairs = ctx->d_stats + 5, *d_ckeep = ctx->d_stats + 6;
    unsigned long long *d_units = ctx->d_stats + 7;
    const float4 *cones = (const float4 *)w_cones;

    // ---- per (light, Gaussian) records, level A: super-tiles ----
    const int nc = n_tiles + n_super;
    rect_cones_kernel<<<(nc + 127) / 128, 128, 0, s>>>(H, W, tile, tx, ty, sx, sy, (float4 *)w_cones,
                                                        p.atlas_map);
    const int grid = (int)std::min<int64_t>((LN + 255) / 256, (int64_t)ctx->num_sms * 16);
    prep_kernel<<<grid, 256, 0, s>>>(means, scales, quats, opac, N, lights, L, radii, K, p.kappa,
                                     p.eps_cull, build_records ? (BuildRec *)w_br : nullptr,
                                     (BinRec *)w_bin, ctx->d_status, roi ? roi->krange : nullptr,
                                     p.beta_mode == 4 ? 3 : p.beta_mode);
    const float4 *scones2 = cones + 2 * (n_tiles + n_super) + PLANE_F4 * n_tiles;
    const bool two = p.atlas_map == MAP_CUBE;
    int64_t capC = p.max_pairs;
    uint32_t *cvals = nullptr;
    if (!want_keys && n_super <= 64) {
        // the build: super-tile masks, per-block ranges, no sort
        void *w_mask, *w_kc;
        if ((rc = ws_reserve(ctx, WS_SMASK, sizeof(unsigned long long) * (size_t)LN, &w_mask))) return rc;
        if ((rc = ws_reserve(ctx, WS_KCNT, 2 * sizeof(uint32_t) * (size_t)nskeys, &w_kc))) return rc;
        uint32_t *kcnt = (uint32_t *)w_kc, *kcur = kcnt + nskeys;
        e = cudaMemsetAsync(kcnt, 0, sizeof(uint32_t) * (size_t)nskeys, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "build: memset");
        (two ? coarse_mask_kernel<true> : coarse_mask_kernel<false>)<<<grid, 256, sizeof(uint32_t) * nskeys, s>>>(
            (const BinRec *)w_bin, N, L, n_super, cones + 2 * n_tiles, scones2, (unsigned long long *)w_mask, kcnt,
            roi ? roi->sact : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "prep/coarse count kernels");
        if ((rc = scan_exclusive_u32(ctx, kcnt, cs, nskeys, d_cpairs, s))) return rc;
        if (capC == 0) {
            unsigned long long Pc;
            if ((rc = read_count(ctx, d_cpairs, s, &Pc))) return rc;
            if (Pc >= (1ull << 31)) return fail(ctx, DGSM_ERR_WORKSPACE, "more than 2^31 (super-tile, Gaussian) pairs");
            if (Pc == 0) return DGSM_OK;
            capC = (int64_t)Pc;
        }
        void *cva;
        if ((rc = ws_reserve(ctx, WS_CVALS_A, sizeof(uint32_t) * capC, &cva))) return rc;
        keep_pairs_kernel<<<1, 32, 0, s>>>(d_cpairs, (unsigned long long)capC, d_ckeep, ctx->d_status);
        key_ranges_kernel<<<(int)((nskeys + 255) / 256), 256, 0, s>>>(kcnt, (int)nskeys, d_ckeep, cs, ce, kcur);
        coarse_scatter_kernel<<<grid, 256, 2 * sizeof(uint32_t) * nskeys, s>>>(
            (const unsigned long long *)w_mask, N, L, n_super, kcur, (uint32_t *)cva, d_ckeep, (uint32_t)capC);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "coarse scatter kernels");
        cvals = (uint32_t *)cva;
    } else {
        // dgsm_bin (and super-tile grids beyond 64 per light): lists sorted by key
        // and, within a key, by Gaussian, as dgsm_bin reports them
        (two ? coarse_bin_kernel<false, true> : coarse_bin_kernel<false, false>)<<<grid, 256, 0, s>>>(
            (const BinRec *)w_bin, N, L, n_super, cones + 2 * n_tiles, scones2, (uint32_t *)w_cnt, nullptr, nullptr,
            nullptr, nullptr, 0u, roi ? roi->sact : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "prep/coarse count kernels");
        if ((rc = scan_exclusive_u32(ctx, (uint32_t *)w_cnt, (uint32_t *)w_cnt, LN, d_cpairs, s))) return rc;
        if (capC == 0) {
            unsigned long long Pc;
            if ((rc = read_count(ctx, d_cpairs, s, &Pc))) return rc;
            if (Pc >= (1ull << 31)) return fail(ctx, DGSM_ERR_WORKSPACE, "more than 2^31 (super-tile, Gaussian) pairs");
            if (Pc == 0) return DGSM_OK;
            capC = (int64_t)Pc;
        }
        void *cka, *cva, *ckb, *cvb;
        if ((rc = ws_reserve(ctx, WS_CKEYS_A, sizeof(uint32_t) * capC, &cka))) return rc;
        if ((rc = ws_reserve(ctx, WS_CVALS_A, sizeof(uint32_t) * capC, &cva))) return rc;
        if ((rc = ws_reserve(ctx, WS_CKEYS_B, sizeof(uint32_t) * capC, &ckb))) return rc;
        if ((rc = ws_reserve(ctx, WS_CVALS_B, sizeof(uint32_t) * capC, &cvb))) return rc;
        keep_pairs_kernel<<<1, 32, 0, s>>>(d_cpairs, (unsigned long long)capC, d_ckeep, ctx->d_status);
        (two ? coarse_bin_kernel<true, true> : coarse_bin_kernel<true, false>)<<<grid, 256, 0, s>>>(
            (const BinRec *)w_bin, N, L, n_super, cones + 2 * n_tiles, scones2, nullptr, (const uint32_t *)w_cnt,
            (uint32_t *)cka, (uint32_t *)cva, d_ckeep, (uint32_t)capC, roi ? roi->sact : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "coarse emit kernel");
        uint32_t *ckeys = (uint32_t *)cka;
        cvals = (uint32_t *)cva;
        if ((rc = radix_sort_pairs(ctx, &ckeys, &cvals, (uint32_t *)ckb, (uint32_t *)cvb, d_ckeep, capC,
                                   key_bits(nskeys), s)))
            return rc;
        const int rgrid = (int)std::min<int64_t>((capC + 255) / 256, (int64_t)ctx->num_sms * 16);
        tile_ranges_kernel<<<rgrid, 256, 0, s>>>(ckeys, d_ckeep, (uint32_t)nskeys, cs, ce);
    }

    // ---- work units of level B ----
    const int64_t max_units = capC / UNIT_G + nskeys + 1;
    void *w_units, *w_fcnt, *w_foff;
    const size_t ucnt_bytes = (sizeof(uint32_t) * (size_t)nskeys + 15) & ~(size_t)15;
    if ((rc = ws_reserve(ctx, WS_UNITS, ucnt_bytes + sizeof(Unit) * (size_t)max_units, &w_units))) return rc;
    uint32_t *ucnt = (uint32_t *)w_units;
    Unit *units = (Unit *)((char *)w_units + ucnt_bytes);
    const int kgrid = (int)((nskeys + 255) / 256);
    unit_count_kernel<<<kgrid, 256, 0, s>>>(cs, ce, (int)nskeys, ucnt);
    if ((rc = scan_exclusive_u32(ctx, ucnt, ucnt, nskeys, d_units, s))) return rc;
    unit_fill_kernel<<<kgrid, 256, 0, s>>>(cs, ce, (int)nskeys, ucnt, units);
    const size_t nf = 64 * (size_t)max_units;
    if ((rc = ws_reserve(ctx, WS_FCNT, sizeof(uint32_t) * nf, &w_fcnt))) return rc;
    if ((rc = ws_reserve(ctx, WS_FOFF, sizeof(uint32_t) * nf, &w_foff))) return rc;
    e = cudaMemsetAsync(w_fcnt, 0, sizeof(uint32_t) * nf, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: memset");
    // many more blocks than fit at once: units differ in cost, and the block
    // scheduler balances them (binning 2.70 ms with 8 blocks per SM, 2.45 with 64)
    const int fgrid = (int)std::min<int64_t>(max_units, (int64_t)ctx->num_sms * 64);
    void *w_fmask;
    if ((rc = ws_reserve(ctx, WS_FMASK, sizeof(uint32_t) * 3 * MASK_WORDS * nf, &w_fmask))) return rc;
    fine_count_kernel<<<fgrid, 256, 0, s>>>(units, d_units, cvals, (const BinRec *)w_bin, N, tx, ty, sx, n_tiles,
                                            n_super, cones, (uint32_t *)w_fcnt, (uint32_t *)w_fmask,
                                            roi ? roi->tact : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fine count kernel");
    if ((rc = scan_exclusive_u32(ctx, (uint32_t *)w_fcnt, (uint32_t *)w_foff, (int64_t)nf, d_pairs, s)))
        return rc;
    int64_t cap = p.max_pairs;
    if (cap == 0) {
        unsigned long long P;
        if ((rc = read_count(ctx, d_pairs, s, &P))) return rc;
        if (P >= (1ull << 31)) return fail(ctx, DGSM_ERR_WORKSPACE, "more than 2^31 binned pairs");
        if (P == 0) return DGSM_OK;
        cap = (int64_t)P;
    }
    out->P = cap;
    void *va, *ka = nullptr;
    if ((rc = ws_reserve(ctx, WS_VALS_A, sizeof(uint32_t) * cap, &va))) return rc;
    if (want_keys && (rc = ws_reserve(ctx, WS_KEYS_A, sizeof(uint32_t) * cap, &ka))) return rc;
    keep_pairs_kernel<<<1, 32, 0, s>>>(d_pairs, (unsigned long long)cap, d_keep, ctx->d_status);
    fine_emit_kernel<<<fgrid, 256, 0, s>>>(units, d_units, cvals, tx, ty, sx, n_tiles, n_super,
                                           (const uint32_t *)w_fmask, (const uint32_t *)w_foff, (uint32_t *)va,
                                           (uint32_t *)ka, d_keep, (uint32_t)cap);
    const int ugrid = (int)std::min<int64_t>((int64_t)((nf + 255) / 256), (int64_t)ctx->num_sms * 16);
    fine_ranges_kernel<<<ugrid, 256, 0, s>>>(units, d_units, (const uint32_t *)w_fcnt,
                                              (const uint32_t *)w_foff, d_keep, n_super, sx, tx, ty,
                                              n_tiles, out->ts, out->te);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fine emit kernels");
    out->keys = (uint32_t *)ka;
    out->vals = (uint32_t *)va;
    return DGSM_OK;
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

namespace dgsm {
namespace {
int check_build(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                const float *opac, int64_t n, const float *lights, int32_t L, int32_t H, int32_t W,
                const float *radii, int32_t K, const dgsm_params &p, void *atlas) {
    int rc = check_common(ctx, means, scales, opac, n, lights, L, H, W, radii, K, p);
    if (rc) return rc;
    if (p.tile == 4) return fail(ctx, DGSM_ERR_INVALID_ARG, "dgsm_build supports tile 8 or 16");
    if (n > 0 && !quats) return fail(ctx, DGSM_ERR_INVALID_ARG, "null quats");
    if (!atlas) return fail(ctx, DGSM_ERR_INVALID_ARG, "null atlas");
    if (p.atlas_dtype < DGSM_F32 || p.atlas_dtype > DGSM_BF16)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "atlas_dtype must be DGSM_F32, DGSM_F16 or DGSM_BF16");
    if (build_smem_bytes(K, p.tile, p.chunk) > 220 * 1024)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "K x tile^2 too large for shared memory: use tile 8");
    if (p.max_pairs < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "max_pairs < 0");
    return DGSM_OK;
}

// The build proper (arguments checked, device current); roi (or nullptr)
// restricts it to a region of interest.
int build_impl(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
               const float *opac, int64_t n, const float *lights, int32_t L, int32_t H, int32_t W,
               const float *radii, int32_t K, const dgsm_params &p, void *atlas, cudaStream_t s,
               const RoiDev *roi) {
    int rc;
    cudaError_t e;
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap_st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamIsCapturing");
    const bool capturing = cap_st != cudaStreamCaptureStatusNone;
    if (capturing && p.max_pairs == 0)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "dgsm_build under stream capture needs max_pairs > 0");
    const bool prof = ctx->prof && !capturing && ctx->prof_count < dgsm_ctx::PROF_RING;
    cudaEvent_t *ev = prof ? ctx->prof_ev[ctx->prof_count] : nullptr;
    if (prof) cudaEventRecord(ev[0], s);
    BinOut b;
    if ((rc = run_binning(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, true, false, s,
                          &b, roi)))
        return rc;

    // ---- work items: every tile's list cut into pieces of <= item Gaussians ----
    const int nkeys = L * b.n_tiles;
    const uint32_t item = (uint32_t)(ITEM_CHUNKS * p.chunk);
    const int64_t max_items = nkeys + b.P / item + 1;
    void *w_items, *w_acc, *w_done;
    const size_t items_bytes = sizeof(Item) * (size_t)max_items + sizeof(uint32_t) * (size_t)nkeys +
                               4 * sizeof(unsigned long long);
    if ((rc = ws_reserve(ctx, WS_ITEMS, items_bytes, &w_items))) return rc;
    const size_t acc_bytes = sizeof(float) * (size_t)L * K * H * W;
    const bool acc_new = ctx->ws_cap[WS_ACCUM] < acc_bytes;
    if ((rc = ws_reserve(ctx, WS_ACCUM, acc_bytes, &w_acc))) return rc;
    const bool done_new = ctx->ws_cap[WS_DONE] < sizeof(uint32_t) * (size_t)nkeys;
    if ((rc = ws_reserve(ctx, WS_DONE, sizeof(uint32_t) * (size_t)nkeys, &w_done))) return rc;
    // the accumulators and counters are returned to zero by the kernel that
    // consumes them; they only need clearing when freshly allocated
    if (acc_new) e = cudaMemsetAsync(w_acc, 0, ctx->ws_cap[WS_ACCUM], s);
    if (e == cudaSuccess && done_new) e = cudaMemsetAsync(w_done, 0, ctx->ws_cap[WS_DONE], s);
    Item *items = (Item *)w_items;
    uint32_t *item_cnt = (uint32_t *)(items + max_items);
    // two 8-byte-aligned counters after the per-key item counts
    unsigned long long *n_items_dev =
        (unsigned long long *)(((uintptr_t)(item_cnt + nkeys) + 7) & ~(uintptr_t)7);
    unsigned int *counter = (unsigned int *)(n_items_dev + 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: item memset");
    item_count_kernel<<<(nkeys + 255) / 256, 256, 0, s>>>(b.ts, b.te, nkeys, item, item_cnt);
    if ((rc = scan_exclusive_u32(ctx, item_cnt, item_cnt, nkeys, n_items_dev, s))) return rc;
    item_expand_kernel<<<(nkeys + 255) / 256, 256, 0, s>>>(b.ts, b.te, nkeys, item, item_cnt, items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: item kernels");
    if (prof) cudaEventRecord(ev[1], s);
    const uint32_t *vals = b.vals ? b.vals : b.ts;  // unused when there are no pairs
    switch (p.atlas_dtype) {
        case DGSM_F32:
            rc = launch_build_items<float>(ctx, b.brec, vals, items, n_items_dev, counter, radii, K,
                                           H, W, p.tile, b.tx, b.n_tiles, n, p.chunk,
                                           (float *)w_acc, (unsigned *)w_done, atlas, s,
                                           roi ? roi->mask : nullptr, roi ? roi->krange : nullptr, p.atlas_map);
            break;
        case DGSM_F16:
            rc = launch_build_items<__half>(ctx, b.brec, vals, items, n_items_dev, counter, radii,
                                            K, H, W, p.tile, b.tx, b.n_tiles, n, p.chunk,
                                            (float *)w_acc, (unsigned *)w_done, atlas, s,
                                            roi ? roi->mask : nullptr, roi ? roi->krange : nullptr, p.atlas_map);
            break;
        default:
            rc = launch_build_items<__nv_bfloat16>(ctx, b.brec, vals, items, n_items_dev, counter,
                                                   radii, K, H, W, p.tile, b.tx, b.n_tiles, n,
                                                   p.chunk, (float *)w_acc, (unsigned *)w_done,
                                                   atlas, s, roi ? roi->mask : nullptr,
                                                   roi ? roi->krange : nullptr, p.atlas_map);
    }
    if (rc) return rc;
    if (prof) {
        cudaEventRecord(ev[2], s);
        ++ctx->prof_count;
    }
    return DGSM_OK;
}

// ---- receiver-driven region of interest (Sec. 3.2, "Receiver-driven ROI") ----

__global__ void roi_init_kernel(int *__restrict__ krange, int L, int K) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) {
        krange[2 * l] = K;
        krange[2 * l + 1] = -1;
    }
}

// Receivers whose centres lie in the box B = {|x - c_x| <= R, |y - c_y| <= R,
// z_min <= z <= z_max} (single-precision decisions) mark, per light, the
// texels and shells their trilinear lookup reads (Sec. 3.3): the 2 x 2
// bilinear taps around their octahedral coordinate and the two shells that
// bracket their distance, both clamped as the lookup clamps them.  The
// marked texels form P; the shells give [k_min, k_max].
__global__ void __launch_bounds__(256) roi_mark_kernel(
    const float *__restrict__ recv, int64_t n, const float *__restrict__ box,
    const float *__restrict__ lights, int L, int H, int W, const float *__restrict__ radii, int K,
    uint8_t *__restrict__ mask, int *__restrict__ krange, int map) {
    __shared__ int skmin[64], skmax[64];
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        skmin[l] = K;
        skmax[l] = -1;
    }
    __syncthreads();
    const float cx = box[0], cy = box[1], R = box[2], z0 = box[3], z1 = box[4];
    const int64_t HW = (int64_t)H * W;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float x = recv[3 * q], y = recv[3 * q + 1], z = recv[3 * q + 2];
        if (!(fabsf(xsub(x, cx)) <= R && fabsf(xsub(y, cy)) <= R && z >= z0 && z <= z1)) continue;
        for (int l = 0; l < L; ++l) {
            const SampleIndex si =
                map == MAP_CUBE ? sample_index_cube(x, y, z, lights[3 * l], lights[3 * l + 1], lights[3 * l + 2], W,
                                                    radii, K, nullptr, ShellTab{})
                                : sample_index(x, y, z, lights[3 * l], lights[3 * l + 1], lights[3 * l + 2], H, W,
                                               radii, K);
            if (si.t == 0.0f) continue;  // at the light: T = 1 without a lookup
            const int j0 = min(max(si.bj, 0), W - 1), j1 = min(max(si.bj + 1, 0), W - 1);
            const int rlo = si.r0, rhi = si.r0 + si.hf - 1;
            const int i0 = min(max(si.bi, rlo), rhi), i1 = min(max(si.bi + 1, rlo), rhi);
            uint8_t *m = mask + l * HW;
            m[(int64_t)i0 * W + j0] = 1;
            m[(int64_t)i0 * W + j1] = 1;
            m[(int64_t)i1 * W + j0] = 1;
            m[(int64_t)i1 * W + j1] = 1;
            const int k0 = si.k < 0 ? 0 : min(si.k, K - 1);
            const int k1 = si.k < 0 ? 0 : min(si.k + 1, K - 1);
            atomicMin(&skmin[l], k0);
            atomicMax(&skmax[l], k1);
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        if (skmax[l] >= 0) {
            atomicMin(&krange[2 * l], skmin[l]);
            atomicMax(&krange[2 * l + 1], skmax[l]);
        }
    }
}

// tact[l][t] = 1 if tile t (tile x tile texels) holds a texel of P.
__global__ void roi_tiles_kernel(const uint8_t *__restrict__ mask, int L, int H, int W, int tile, int tx,
                                 int n_tiles, uint8_t *__restrict__ tact) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * n_tiles) return;
    const int l = (int)(idx / n_tiles), t = (int)(idx - (int64_t)l * n_tiles);
    const int ti = t / tx, tj = t - ti * tx;
    const uint8_t *m = mask + (int64_t)l * H * W;
    uint8_t any = 0;
    for (int i = ti * tile; i < min((ti + 1) * tile, H) && !any; ++i)
        for (int j = tj * tile; j < min((tj + 1) * tile, W); ++j) any |= m[(int64_t)i * W + j];
    tact[idx] = any;
}

// sact[l][s] = 1 if super-tile s (SUPER x SUPER tiles) holds an active tile.
__global__ void roi_super_kernel(const uint8_t *__restrict__ tact, int L, int tx, int ty, int sx,
                                 int n_tiles, int n_super, uint8_t *__restrict__ sact) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L * n_super) return;
    const int l = (int)(idx / n_super), sidx = (int)(idx - (int64_t)l * n_super);
    const int sa = sidx / sx, sb = sidx - sa * sx;
    uint8_t any = 0;
    for (int a = sa * SUPER; a < min((sa + 1) * SUPER, ty); ++a)
        for (int b = sb * SUPER; b < min((sb + 1) * SUPER, tx); ++b) any |= tact[(int64_t)l * n_tiles + a * tx + b];
    sact[idx] = any;
}

}  // namespace
}  // namespace dgsm

extern "C" int dgsm_build(dgsm_ctx *ctx, const float *means, const float *scales,
                          const float *quats, const float *opac, int64_t n, const float *lights,
                          int32_t L, int32_t H, int32_t W, const float *radii, int32_t K,
                          const dgsm_params *params, void *atlas, void *stream) {
    DGSM_RANGE("dgsm_build");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    int rc = check_build(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, atlas);
    if (rc) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return build_impl(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, atlas,
                      (cudaStream_t)stream, nullptr);
}

extern "C" int dgsm_build_roi(dgsm_ctx *ctx, const float *means, const float *scales,
                              const float *quats, const float *opac, int64_t n, const float *lights,
                              int32_t L, int32_t H, int32_t W, const float *radii, int32_t K,
                              const dgsm_params *params, const dgsm_roi *roi, void *atlas,
                              void *stream) {
    DGSM_RANGE("dgsm_build_roi");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    int rc = check_build(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, atlas);
    if (rc) return rc;
    if (!roi || !roi->box) return fail(ctx, DGSM_ERR_INVALID_ARG, "null roi or roi box");
    if (roi->n_recv < 0 || (roi->n_recv > 0 && !roi->recv_means))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "bad roi receivers");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int tx = (W + p.tile - 1) / p.tile, ty = (H + p.tile - 1) / p.tile;
    const int sx = (tx + SUPER - 1) / SUPER, sy = (ty + SUPER - 1) / SUPER;
    const int64_t n_tiles = (int64_t)tx * ty, n_super = (int64_t)sx * sy;
    const int64_t HW = (int64_t)H * W;
    const size_t kr_bytes = ((size_t)L * 2 * sizeof(int) + 255) & ~(size_t)255;
    const size_t m_bytes = ((size_t)(L * HW) + 255) & ~(size_t)255;
    const size_t t_bytes = ((size_t)(L * n_tiles) + 255) & ~(size_t)255;
    const size_t total = kr_bytes + m_bytes + t_bytes + (size_t)(L * n_super);
    void *w;
    if ((rc = ws_reserve(ctx, WS_ROI, total, &w))) return rc;
    RoiDev r;
    int *krange = (int *)w;
    uint8_t *mask = (uint8_t *)w + kr_bytes;
    uint8_t *tact = mask + m_bytes, *sact = tact + t_bytes;
    r.krange = krange;
    r.mask = mask;
    r.tact = tact;
    r.sact = sact;
    e = cudaMemsetAsync(mask, 0, (size_t)(L * HW), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "roi: memset");
    roi_init_kernel<<<1, 64, 0, s>>>(krange, L, K);
    if (roi->n_recv > 0) {
        const int grid = (int)std::min<int64_t>((roi->n_recv + 255) / 256, (int64_t)ctx->num_sms * 8);
        roi_mark_kernel<<<grid, 256, 0, s>>>(roi->recv_means, roi->n_recv, roi->box, lights, L, H, W, radii,
                                             K, mask, krange, p.atlas_map);
    }
    roi_tiles_kernel<<<(int)((L * n_tiles + 255) / 256), 256, 0, s>>>(mask, L, H, W, p.tile, tx, (int)n_tiles,
                                                                       tact);
    roi_super_kernel<<<(int)((L * n_super + 255) / 256), 256, 0, s>>>(tact, L, tx, ty, sx, (int)n_tiles,
                                                                       (int)n_super, sact);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "roi kernels");
    if (roi->mask_out) e = cudaMemcpyAsync(roi->mask_out, mask, (size_t)(L * HW), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && roi->krange_out)
        e = cudaMemcpyAsync(roi->krange_out, krange, (size_t)L * 2 * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "roi: copy out");
    return build_impl(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, atlas, s, &r);
}

// ---- a band of atlas rows (the multi-GPU split of one light's atlas) ----

namespace dgsm {
namespace {

// mask[l][i][j] = 1 for rows [row0, row1); every shell in range.
__global__ void band_init_kernel(uint8_t *__restrict__ mask, int *__restrict__ krange, int L, int H, int W, int K,
                                 int row0, int row1) {
    const int64_t HW = (int64_t)H * W;
    const int64_t total = (int64_t)L * HW;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)((idx % HW) / W);
        mask[idx] = i >= row0 && i < row1;
        if (idx < L) {
            krange[2 * idx] = 0;
            krange[2 * idx + 1] = K - 1;
        }
    }
}

}  // namespace
}  // namespace dgsm

extern "C" int dgsm_build_band(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                               const float *opac, int64_t n, const float *lights, int32_t L, int32_t H,
                               int32_t W, const float *radii, int32_t K, const dgsm_params *params,
                               int32_t row0, int32_t row1, void *atlas, void *stream) {
    DGSM_RANGE("dgsm_build_band");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    int rc = check_build(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, atlas);
    if (rc) return rc;
    if (!(0 <= row0 && row0 < row1 && row1 <= H))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "band rows: need 0 <= row0 < row1 <= H");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int tx = (W + p.tile - 1) / p.tile, ty = (H + p.tile - 1) / p.tile;
    const int sx = (tx + SUPER - 1) / SUPER, sy = (ty + SUPER - 1) / SUPER;
    const int64_t n_tiles = (int64_t)tx * ty, n_super = (int64_t)sx * sy;
    const int64_t HW = (int64_t)H * W;
    const size_t kr_bytes = ((size_t)L * 2 * sizeof(int) + 255) & ~(size_t)255;
    const size_t m_bytes = ((size_t)(L * HW) + 255) & ~(size_t)255;
    const size_t t_bytes = ((size_t)(L * n_tiles) + 255) & ~(size_t)255;
    const size_t total = kr_bytes + m_bytes + t_bytes + (size_t)(L * n_super);
    void *w;
    if ((rc = ws_reserve(ctx, WS_ROI, total, &w))) return rc;
    RoiDev r;
    int *krange = (int *)w;
    uint8_t *mask = (uint8_t *)w + kr_bytes;
    uint8_t *tact = mask + m_bytes, *sact = tact + t_bytes;
    r.krange = krange;
    r.mask = mask;
    r.tact = tact;
    r.sact = sact;
    const int grid = (int)std::min<int64_t>((L * HW + 255) / 256, (int64_t)ctx->num_sms * 8);
    band_init_kernel<<<grid, 256, 0, s>>>(mask, krange, L, H, W, K, row0, row1);
    roi_tiles_kernel<<<(int)((L * n_tiles + 255) / 256), 256, 0, s>>>(mask, L, H, W, p.tile, tx, (int)n_tiles,
                                                                       tact);
    roi_super_kernel<<<(int)((L * n_super + 255) / 256), 256, 0, s>>>(tact, L, tx, ty, sx, (int)n_tiles,
                                                                       (int)n_super, sact);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band kernels");
    return build_impl(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, atlas, s, &r);
}

extern "C" int dgsm_atlas_rows_copy(dgsm_ctx *ctx, const void *src, int32_t src_rows, int32_t src_row0, void *dst,
                                    int32_t dst_rows, int32_t dst_row0, int32_t rows, int64_t planes, int32_t W,
                                    int32_t elem_bytes, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (rows == 0 || planes == 0) return DGSM_OK;
    if (!src || !dst || rows < 0 || planes < 0 || W < 1 || (elem_bytes != 2 && elem_bytes != 4) ||
        src_row0 < 0 || dst_row0 < 0 || src_row0 + rows > src_rows || dst_row0 + rows > dst_rows)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "atlas rows copy: rows out of range or bad sizes");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const size_t row_b = (size_t)W * elem_bytes;
    e = cudaMemcpy2DAsync((char *)dst + (size_t)dst_row0 * row_b, (size_t)dst_rows * row_b,
                          (const char *)src + (size_t)src_row0 * row_b, (size_t)src_rows * row_b,
                          (size_t)rows * row_b, (size_t)planes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "atlas rows copy");
}

extern "C" int dgsm_get_build_stats(dgsm_ctx *ctx, dgsm_build_stats *out) {
    if (!ctx || !out) return DGSM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(ctx->h_pinned + 4, ctx->d_stats, 6 * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dgsm_get_build_stats");
    out->n_pairs = (int64_t)ctx->h_pinned[7];
    out->rays_tested = (int64_t)ctx->h_pinned[4];
    out->ray_evals = (int64_t)ctx->h_pinned[5];
    out->shell_evals = (int64_t)ctx->h_pinned[6];
    out->n_super_pairs = (int64_t)ctx->h_pinned[9];
    return DGSM_OK;
}

extern "C" int dgsm_bin(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                        const float *opac, int64_t n, const float *lights, int32_t L, int32_t H,
                        int32_t W, const float *radii, int32_t K, const dgsm_params *params,
                        uint32_t *keys_out, uint32_t *vals_out, int64_t capacity,
                        int64_t *n_pairs_out, void *stream) {
    DGSM_RANGE("dgsm_bin");
    if (!ctx || !n_pairs_out) return DGSM_ERR_INVALID_ARG;
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    p.max_pairs = 0;  // exact count: it is returned to the caller
    int rc = check_common(ctx, means, scales, opac, n, lights, L, H, W, radii, K, p);
    if (rc) return rc;
    if (capacity < 0 || (capacity > 0 && (!keys_out || !vals_out)))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "bad output capacity or pointers");
    if (n > 0 && !quats) return fail(ctx, DGSM_ERR_INVALID_ARG, "null quats");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    BinOut b;
    if ((rc = run_binning(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, false, true, s,
                          &b)))
        return rc;
    *n_pairs_out = b.P;
    if (b.P > capacity) return fail(ctx, DGSM_ERR_WORKSPACE, "capacity smaller than the pair count");
    if (b.P > 0) {
        // the pairs are laid out super-tile by super-tile: sort them by key
        // (stable, so each key keeps its Gaussian order)
        void *kb, *vb;
        if ((rc = ws_reserve(ctx, WS_KEYS_B, sizeof(uint32_t) * b.P, &kb))) return rc;
        if ((rc = ws_reserve(ctx, WS_VALS_B, sizeof(uint32_t) * b.P, &vb))) return rc;
        uint32_t *keys = b.keys, *vals = b.vals;
        if ((rc = radix_sort_pairs(ctx, &keys, &vals, (uint32_t *)kb, (uint32_t *)vb, ctx->d_stats + 4, b.P,
                                   key_bits((int64_t)L * b.n_tiles), s)))
            return rc;
        e = cudaMemcpyAsync(keys_out, keys, sizeof(uint32_t) * b.P, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals_out, vals, sizeof(uint32_t) * b.P, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dgsm_bin copy-out");
    return DGSM_OK;
}
