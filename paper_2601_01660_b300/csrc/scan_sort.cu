// scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort
// (the prefix sums and the sort of the light-space tile binning).
#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // items per block

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total.  blockDim.x must be a multiple of 32
// and at most 1024.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total) {
    __shared__ T warp_sums[33];  // [32] holds the block total
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_sums[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == nw - 1) warp_sums[32] = wi;
    }
    __syncthreads();
    T res = warp_sums[warp] + inc - v;
    *total = warp_sums[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const uint32_t *__restrict__ in,
                                                                   int64_t n,
                                                                   unsigned long long *block_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    unsigned long long acc = 0;
    for (int e = threadIdx.x; e < SCAN_TILE; e += SCAN_THREADS) {
        int64_t i = base + e;
        if (i < n) acc += in[i];
    }
    unsigned long long tot;
    block_exclusive_scan(acc, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// One block of 1024 threads scans the block sums in place (exclusive).
__global__ void __launch_bounds__(1024) scan_blocks_kernel(unsigned long long *block_sums, int64_t nb,
                                                           unsigned long long *d_total) {
    unsigned long long carry = 0;
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        unsigned long long v = i < nb ? block_sums[i] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_exclusive_scan(v, &tot);
        if (i < nb) block_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_apply_kernel(const uint32_t *in, uint32_t *out,
                                                                  int64_t n,
                                                                  const unsigned long long *block_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    unsigned long long sum = 0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        v[e] = base + e < n ? in[base + e] : 0u;
        sum += v[e];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_scan(sum, &tot) + block_sums[blockIdx.x];
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        if (base + e < n) out[base + e] = (uint32_t)run;
        run += v[e];
    }
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits; one block sorts a segment of 16 rounds x 256
// items.  Stability comes from ranking each round's items in thread order
// (warp match + per-warp digit counts) on top of the running digit counts;
// the segment is ordered in shared memory and written out run by run.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_SEG = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) radix_hist_kernel(const uint32_t *__restrict__ keys,
                                                                const unsigned long long *d_n, int shift,
                                                                uint32_t *__restrict__ hist, int nb) {
    __shared__ uint32_t h[256];
    const int64_t n = (int64_t)*d_n;
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_SEG;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) radix_scatter_kernel(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
    const unsigned long long *d_n, int shift, const uint32_t *__restrict__ offs, int nb) {
    // The block's segment is first put in digit order in shared memory (each
    // round's items ranked in thread order on top of the running digit
    // counts), then written out: consecutive threads write consecutive items
    // of one digit's run, so the stores coalesce.
    __shared__ uint32_t gbase[256];   // global start of each digit's run of this block
    __shared__ uint32_t lstart[256];  // start of each digit's run in the block's order
    __shared__ uint32_t lrun[256];    // items of each digit placed so far
    __shared__ uint32_t wsum[RS_WARPS];
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t sk[RS_SEG], sv[RS_SEG];
    const int64_t n = (int64_t)*d_n;
    const int64_t seg = (int64_t)blockIdx.x * RS_SEG;
    if (seg >= n) return;  // uniform across the block
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // offsets are digit-major ([digit][block]), so the block's count of digit
    // tid is the next entry minus this one (the total n after the last)
    const int64_t e = (int64_t)tid * nb + blockIdx.x;
    const uint32_t o = offs[e];
    const uint32_t c = (tid == 255 && blockIdx.x == nb - 1 ? (uint32_t)n : offs[e + 1]) - o;
    gbase[tid] = o;
    uint32_t x = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += wsum[w];
    lstart[tid] = x - c + add;
    lrun[tid] = 0;
    const int seg_n = (int)min((int64_t)RS_SEG, n - seg);
    for (int r = 0; r < RS_ROUNDS; ++r) {
        if (r * RS_THREADS >= seg_n) break;  // uniform across the block
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int li = r * RS_THREADS + tid;
        const bool valid = li < seg_n;
        const uint32_t k = valid ? keys_in[seg + li] : 0u;
        const uint32_t v = valid ? vals_in[seg + li] : 0u;
        const int d = valid ? (int)((k >> shift) & 255u) : 256 + lane;
        const unsigned m = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(m & lt_mask);
        if (valid && lane == __ffs(m) - 1) wcnt[warp][d] = __popc(m);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t cw = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += cw;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = lstart[d] + lrun[d] + wcnt[warp][d] + (uint32_t)rank;
            sk[pos] = k;
            sv[pos] = v;
        }
        __syncthreads();
        lrun[tid] += run;
    }
    __syncthreads();
    for (int i = tid; i < seg_n; i += RS_THREADS) {
        const uint32_t k = sk[i];
        const int d = (int)((k >> shift) & 255u);
        const uint32_t dst = gbase[d] + ((uint32_t)i - lstart[d]);
        keys_out[dst] = k;
        vals_out[dst] = sv[i];
    }
}

}  // namespace

int scan_exclusive_u32(dgsm_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n,
                       unsigned long long *d_total, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) {
            cudaError_t e = cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "scan: memset");
        }
        return DGSM_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    void *tmp;
    int rc = ws_reserve(ctx, WS_SCAN_TMP, sizeof(unsigned long long) * nb, &tmp);
    if (rc) return rc;
    unsigned long long *bs = (unsigned long long *)tmp;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bs);
    scan_blocks_kernel<<<1, 1024, 0, s>>>(bs, nb, d_total);
    scan_apply_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, bs);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "scan kernels");
}

int radix_sort_pairs(dgsm_ctx *ctx, uint32_t **keys_io, uint32_t **vals_io, uint32_t *keys_alt,
                     uint32_t *vals_alt, const unsigned long long *d_n, int64_t n_max, int bits,
                     cudaStream_t s) {
    if (n_max <= 1 || bits <= 0) return DGSM_OK;
    int nb = (int)((n_max + RS_SEG - 1) / RS_SEG);
    void *h;
    int rc = ws_reserve(ctx, WS_HIST, sizeof(uint32_t) * 256 * (size_t)nb, &h);
    if (rc) return rc;
    uint32_t *hist = (uint32_t *)h;
    uint32_t *ka = *keys_io, *va = *vals_io, *kb = keys_alt, *vb = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_kernel<<<nb, RS_THREADS, 0, s>>>(ka, d_n, shift, hist, nb);
        rc = scan_exclusive_u32(ctx, hist, hist, 256 * (int64_t)nb, nullptr, s);
        if (rc) return rc;
        radix_scatter_kernel<<<nb, RS_THREADS, 0, s>>>(ka, va, kb, vb, d_n, shift, hist, nb);
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    *keys_io = ka;
    *vals_io = va;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "radix sort kernels");
}

}  // namespace dgsm
