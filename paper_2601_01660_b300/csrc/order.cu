// order.cu -- the spatial (Z-order) storage order of a scene's Gaussians.
//
// Every per-Gaussian result of the method (a build record, a binning
// decision, an attenuation or relight of one receiver) is independent of the
// Gaussian's place in the arrays; only the order of the floating-point sums
// into an atlas voxel changes with it.  Storing a scene in the Z-order of its
// means makes consecutive Gaussians neighbours in space, hence in direction
// from any light: the atlas taps of a warp of receivers (Sec. 3.3) then fall
// in a few sectors instead of one or two per lane.  The order is taken once,
// when a scene is loaded; dgsm_gather_rows applies it to each attribute.
#include <algorithm>
#include <cstdint>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int ORD_THREADS = 256;

// Monotone map of floats to unsigned integers (the IEEE order, -0 < +0).
__device__ __forceinline__ uint32_t ord_of(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// box[0..2]: ord_of of the smallest x, y, z; box[3..5]: of the largest
// (box preset to 0xffffffff / 0 by the caller); *d_n = n.
__global__ void __launch_bounds__(ORD_THREADS) ord_box_kernel(const float *__restrict__ means, int64_t n,
                                                              uint32_t *__restrict__ box,
                                                              unsigned long long *__restrict__ d_n) {
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const uint32_t o = ord_of(means[3 * i + a]);
            lo[a] = min(lo[a], o);
            hi[a] = max(hi[a], o);
        }
    for (int a = 0; a < 3; ++a)
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(box + a, lo[a]);
            atomicMax(box + 3 + a, hi[a]);
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = (unsigned long long)n;
}

// 10 bits per axis, interleaved x, y, z from the lowest bit up.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// keys[i]: the Z-order code of mean i on a 1024^3 grid over the box: cell
// q_a = floor((x_a - lo_a) * (1024 / (hi_a - lo_a))) clamped to [0, 1023],
// every operation rounded once (no contraction), so that the codes can be
// recomputed bit for bit elsewhere; a flat axis (hi = lo) has q_a = 0.
__global__ void __launch_bounds__(ORD_THREADS) ord_key_kernel(const float *__restrict__ means, int64_t n,
                                                              const uint32_t *__restrict__ box,
                                                              uint32_t *__restrict__ keys,
                                                              uint32_t *__restrict__ vals) {
    float lo[3], inv[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = float_of(box[a]);
        const float ext = __fsub_rn(float_of(box[3 + a]), lo[a]);
        inv[a] = ext > 0.0f ? __fdiv_rn(1024.0f, ext) : 0.0f;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t code = 0u;
        for (int a = 0; a < 3; ++a) {
            const float f = floorf(__fmul_rn(__fsub_rn(means[3 * i + a], lo[a]), inv[a]));
            const uint32_t q = (uint32_t)fminf(fmaxf(f, 0.0f), 1023.0f);  // NaN -> 0
            code |= spread3(q) << a;
        }
        keys[i] = code;
        vals[i] = (uint32_t)i;
    }
}

// dst row i = src row perm[i], rows of `words` 32-bit words; consecutive
// threads take consecutive words of dst.  A perm entry outside [0, n_src)
// leaves its row zero and records DGSM_ERR_INVALID_ARG in the status word.
__global__ void __launch_bounds__(ORD_THREADS) gather_rows_kernel(const uint32_t *__restrict__ src,
                                                                  int64_t n_src, uint32_t *__restrict__ dst,
                                                                  int64_t words, const int32_t *__restrict__ perm,
                                                                  int64_t n, int *status) {
    const int64_t total = n * words;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / words, w = e - i * words;
        const int64_t r = perm[i];
        if (r < 0 || r >= n_src) {
            dst[e] = 0u;
            if (w == 0) record_status(status, DGSM_ERR_INVALID_ARG);
            continue;
        }
        dst[e] = __ldg(src + r * words + w);
    }
}

unsigned ord_grid(int64_t work, int device) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int64_t need = (work + ORD_THREADS - 1) / ORD_THREADS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_spatial_order(dgsm_ctx *ctx, const float *means, int64_t n, int32_t *perm_out, void *stream) {
    DGSM_RANGE("dgsm_spatial_order");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || n > 0x7fffffffLL) return fail(ctx, DGSM_ERR_INVALID_ARG, "spatial order: 0 <= n < 2^31");
    if (n == 0) return DGSM_OK;
    if (!means || !perm_out) return fail(ctx, DGSM_ERR_INVALID_ARG, "spatial order: null array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t nn = (size_t)n;
    const size_t off_keys = 0, off_vals = 4 * nn, off_keys2 = 8 * nn, off_vals2 = 12 * nn,
                 off_box = (16 * nn + 15) & ~(size_t)15, off_cnt = off_box + 32, total = off_cnt + 16;
    void *w;
    int rc = ws_reserve(ctx, WS_ORDER, total, &w);
    if (rc) return rc;
    char *base = (char *)w;
    uint32_t *keys = (uint32_t *)(base + off_keys), *vals = (uint32_t *)(base + off_vals);
    uint32_t *keys2 = (uint32_t *)(base + off_keys2), *vals2 = (uint32_t *)(base + off_vals2);
    uint32_t *box = (uint32_t *)(base + off_box);
    unsigned long long *d_n = (unsigned long long *)(base + off_cnt);
    e = cudaMemsetAsync(box, 0xff, 12, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(box + 3, 0, 12, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "spatial order: memset");
    const unsigned grid = ord_grid(n, ctx->device);
    ord_box_kernel<<<grid, ORD_THREADS, 0, s>>>(means, n, box, d_n);
    ord_key_kernel<<<grid, ORD_THREADS, 0, s>>>(means, n, box, keys, vals);
    rc = radix_sort_pairs(ctx, &keys, &vals, keys2, vals2, d_n, n, 30, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(perm_out, vals, 4 * nn, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "spatial order: copy");
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "spatial order kernels");
}

extern "C" int dgsm_gather_rows(dgsm_ctx *ctx, const void *src, int64_t n_src, int64_t row_bytes,
                                const int32_t *perm, int64_t n, void *dst, void *stream) {
    DGSM_RANGE("dgsm_gather_rows");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || n_src < 0 || row_bytes <= 0 || (row_bytes & 3) != 0)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "gather rows: n >= 0, row_bytes a positive multiple of 4");
    if (n == 0) return DGSM_OK;
    if (!src || !perm || !dst) return fail(ctx, DGSM_ERR_INVALID_ARG, "gather rows: null array");
    if (src == dst) return fail(ctx, DGSM_ERR_INVALID_ARG, "gather rows: dst must not be src");
    if ((((uintptr_t)src) & 3u) || (((uintptr_t)dst) & 3u))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "gather rows: arrays not 4-byte aligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const int64_t words = row_bytes / 4;
    gather_rows_kernel<<<ord_grid(n * words, ctx->device), ORD_THREADS, 0, (cudaStream_t)stream>>>(
        (const uint32_t *)src, n_src, (uint32_t *)dst, words, perm, n, ctx->d_status);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "gather_rows_kernel");
}
