// sh.cu -- HDRI probe fit (Sec. 3.4, Eq. 7, FP64) and per-Gaussian radiance
// transfer (Sec. 3.5, Eqs. 8-10) on sm_103a.
#include <cuda.h>  // CUcontext, CUresult: two driver functions looked up at run time

#include <algorithm>
#include <mutex>

#include "dgsm_internal.cuh"
#include "relight.cuh"

namespace dgsm {
namespace {

constexpr int FIT_THREADS = 256;
constexpr int FIT_NV = 45 + 27;  // upper triangle of B^T W B, then B^T W Y (9 x 3)

// Per-block FP64 partial sums of the normal equations.
__global__ void __launch_bounds__(FIT_THREADS) sh_fit_partial_kernel(
    const float *__restrict__ dirs, const float *__restrict__ rgb, const float *__restrict__ w,
    int64_t n, double *__restrict__ partials) {
    double acc[FIT_NV];
#pragma unroll
    for (int v = 0; v < FIT_NV; ++v) acc[v] = 0.0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        double Y[9];
        sh9<double>(dirs[3 * s], dirs[3 * s + 1], dirs[3 * s + 2], Y);
        const double ws = w[s];
        int v = 0;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const double wa = ws * Y[a];
#pragma unroll
            for (int b = a; b < 9; ++b) {
                acc[v] = fma(wa, Y[b], acc[v]);
                ++v;
            }
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const double wa = ws * Y[a];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[v] = fma(wa, (double)rgb[3 * s + c], acc[v]);
                ++v;
            }
        }
    }
    __shared__ double red[FIT_THREADS / 32][FIT_NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < FIT_NV; ++v) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][v] = x;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < FIT_NV; v += blockDim.x) {
        double x = 0.0;
        for (int q = 0; q < FIT_THREADS / 32; ++q) x += red[q][v];
        partials[(int64_t)blockIdx.x * FIT_NV + v] = x;
    }
}

// One block: sum the partials in a fixed order, add lambda I, Cholesky-solve.
__global__ void sh_fit_solve_kernel(const double *__restrict__ partials, int nblocks,
                                    double lambda, float *__restrict__ sh_out,
                                    double *__restrict__ sh64_out, int *__restrict__ status) {
    __shared__ double sums[FIT_NV];
    for (int v = threadIdx.x; v < FIT_NV; v += blockDim.x) {
        double x = 0.0;
        for (int b = 0; b < nblocks; ++b) x += partials[(int64_t)b * FIT_NV + v];
        sums[v] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double G[9][9], R[9][3], Lm[9][9];
    int v = 0;
    for (int a = 0; a < 9; ++a)
        for (int b = a; b < 9; ++b) {
            G[a][b] = sums[v];
            G[b][a] = sums[v];
            ++v;
        }
    for (int a = 0; a < 9; ++a)
        for (int c = 0; c < 3; ++c) R[a][c] = sums[v++];
    for (int a = 0; a < 9; ++a) G[a][a] += lambda;
    bool ok = true;
    for (int i = 0; i < 9 && ok; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = G[i][j];
            for (int k = 0; k < j; ++k) s -= Lm[i][k] * Lm[j][k];
            if (i == j) {
                if (!(s > 0.0)) { ok = false; break; }
                Lm[i][i] = sqrt(s);
            } else {
                Lm[i][j] = s / Lm[j][j];
            }
        }
    if (!ok) {
        atomicCAS(status, 0, DGSM_ERR_NOT_SPD);
        for (int k = 0; k < 27; ++k) {
            sh_out[k] = 0.0f;
            if (sh64_out) sh64_out[k] = 0.0;
        }
        return;
    }
    for (int c = 0; c < 3; ++c) {
        double yv[9], xv[9];
        for (int i = 0; i < 9; ++i) {
            double s = R[i][c];
            for (int k = 0; k < i; ++k) s -= Lm[i][k] * yv[k];
            yv[i] = s / Lm[i][i];
        }
        for (int i = 8; i >= 0; --i) {
            double s = yv[i];
            for (int k = i + 1; k < 9; ++k) s -= Lm[k][i] * xv[k];
            xv[i] = s / Lm[i][i];
        }
        for (int k = 0; k < 9; ++k) {
            sh_out[9 * c + k] = (float)xv[k];
            if (sh64_out) sh64_out[9 * c + k] = xv[k];
        }
    }
}

// Radiance transfer.  Each block first tabulates the lat-long quadrature
// (direction, weight w_j, w_j L_c(w_j)) in shared memory, then contracts it
// against the lobe of each of its Gaussians.
constexpr int RELIGHT_G = 4;  // Gaussians per thread in relight_kernel

__global__ void __launch_bounds__(256) relight_kernel(
    const float *__restrict__ sh, const float *__restrict__ means, const float *__restrict__ quats,
    const float *__restrict__ scales, const float *__restrict__ normals,
    const float *__restrict__ centroid, const __grid_constant__ Segs segs, const float *cin,
    int64_t N, float q, float gamma, float t_max, float eps, int nth, int nph, float *cout) {
    extern __shared__ float4 tab[];  // 2 per direction: (omega, w), (w L_r, w L_g, w L_b, 0)
    __shared__ float shs[27];
    __shared__ float cen[3 * MAX_OBJECTS];  // centroid of each object (normals == NULL)
    const int M = nth * nph;
    for (int k = threadIdx.x; k < 27; k += blockDim.x) shs[k] = sh[k];
    if (!normals)
        for (int k = threadIdx.x; k < 3 * segs.n; k += blockDim.x) cen[k] = centroid[k];
    __syncthreads();
    relight_table_fill(shs, 0, M, nth, nph, tab);
    __syncthreads();
    // RELIGHT_G Gaussians per thread, blockDim apart: one read of each table
    // entry serves all of them, which keeps the loop on the FP32 pipe
    const int64_t per_block = (int64_t)blockDim.x * RELIGHT_G;
    for (int64_t base = (int64_t)blockIdx.x * per_block; base < N; base += (int64_t)gridDim.x * per_block) {
        float3 n[RELIGHT_G];
#pragma unroll
        for (int r = 0; r < RELIGHT_G; ++r) {
            const int64_t g = base + r * (int64_t)blockDim.x + threadIdx.x;
            if (g >= N) {
                n[r] = make_float3(0.f, 0.f, 1.f);  // a padding slot: summed, never written
            } else if (normals) {
                n[r] = make_float3(normals[3 * g], normals[3 * g + 1], normals[3 * g + 2]);
                const float inv = rsqrtf(n[r].x * n[r].x + n[r].y * n[r].y + n[r].z * n[r].z);
                n[r].x *= inv; n[r].y *= inv; n[r].z *= inv;
            } else {
                const int o = segs.n == 1 ? 0 : seg_find(segs, g);
                n[r] = relight_axis_normal(means, quats, scales, g, cen[3 * o], cen[3 * o + 1], cen[3 * o + 2]);
            }
        }
        float4 acc[RELIGHT_G];
        relight_accumulate<RELIGHT_G>(tab, M, q, n, acc);
#pragma unroll
        for (int r = 0; r < RELIGHT_G; ++r) {
            const int64_t g = base + r * (int64_t)blockDim.x + threadIdx.x;
            if (g < N) relight_write(acc[r], eps, t_max, gamma, cin, cout, g);
        }
    }
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int sh_fit(dgsm_ctx *ctx, const float *dirs, const float *rgb, const float *w,
                      int64_t n, double lambda, float *sh_out, double *sh64_out, void *stream) {
    DGSM_RANGE("sh_fit");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 1 || !dirs || !rgb || !w || !sh_out) return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_fit: need n >= 1 and non-null arrays");
    if (!(lambda >= 0.0)) return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_fit: lambda must be >= 0");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)std::min<int64_t>((n + FIT_THREADS - 1) / FIT_THREADS, (int64_t)ctx->num_sms);
    void *part;
    int rc = ws_reserve(ctx, WS_SH_PART, sizeof(double) * FIT_NV * nblocks, &part);
    if (rc) return rc;
    sh_fit_partial_kernel<<<nblocks, FIT_THREADS, 0, s>>>(dirs, rgb, w, n, (double *)part);
    sh_fit_solve_kernel<<<1, 128, 0, s>>>((const double *)part, nblocks, lambda, sh_out, sh64_out,
                                          ctx->d_status);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "sh_fit kernels");
}

namespace {
int relight_launch(dgsm_ctx *ctx, const float *sh, const float *means, const float *quats,
                   const float *scales, const float *normals, const float *centroids,
                   const Segs &segs, const float *colors_in, int64_t n,
                   const dgsm_relight_params *params, float *colors_out, void *stream) {
    dgsm_relight_params p;
    if (params) p = *params; else dgsm_default_relight_params(&p);
    if (p.n_theta < 1 || p.n_phi < 1 || (int64_t)p.n_theta * p.n_phi > 6144)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_relight: need 1 <= n_theta * n_phi <= 6144");
    if (!(p.q > 0.0f) || !(p.eps >= 0.0f) || !(p.t_max >= 0.0f))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_relight: need q > 0, eps >= 0, t_max >= 0");
    if (!sh) return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_relight: null sh");
    if (n > 0 && (!colors_in || !colors_out || (!normals && (!means || !quats || !scales || !centroids))))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_relight: null Gaussian array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n == 0) return DGSM_OK;
    const size_t smem = (size_t)p.n_theta * p.n_phi * 2 * sizeof(float4);
    e = cudaFuncSetAttribute(relight_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "relight smem attribute");
    // as many blocks as fit at once (the table decides), at most one group of
    // RELIGHT_G x 256 Gaussians each
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, relight_kernel, 256, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "relight occupancy");
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + 256 * RELIGHT_G - 1) / (256 * RELIGHT_G), (int64_t)ctx->num_sms * std::max(per_sm, 1)));
    relight_kernel<<<grid, 256, smem, (cudaStream_t)stream>>>(
        sh, means, quats, scales, normals, centroids, segs, colors_in, n, p.q, p.gamma, p.t_max,
        p.eps, p.n_theta, p.n_phi, colors_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "relight_kernel");
}
}  // namespace

extern "C" int sh_relight(dgsm_ctx *ctx, const float *sh, const float *means, const float *quats,
                          const float *scales, const float *normals, const float *centroid,
                          const float *colors_in, int64_t n, const dgsm_relight_params *params,
                          float *colors_out, void *stream) {
    DGSM_RANGE("sh_relight");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_relight: n < 0");
    const int64_t whole[2] = {0, n};
    Segs segs;
    make_segs(whole, 1, n, &segs);
    return relight_launch(ctx, sh, means, quats, scales, normals, centroid, segs, colors_in, n,
                          params, colors_out, stream);
}

extern "C" int sh_relight_objects(dgsm_ctx *ctx, const float *sh, const float *means,
                                  const float *quats, const float *scales, const float *centroids,
                                  const int64_t *seg, int32_t n_obj, const float *colors_in,
                                  int64_t n, const dgsm_relight_params *params, float *colors_out,
                                  void *stream) {
    DGSM_RANGE("sh_relight_objects");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "sh_relight_objects: n < 0");
    Segs segs;
    if (!make_segs(seg, n_obj, n, &segs))
        return fail(ctx, DGSM_ERR_INVALID_ARG,
                    "sh_relight_objects: need 1 <= n_obj <= 64 and 0 = seg[0] <= ... <= seg[n_obj] = n");
    return relight_launch(ctx, sh, means, quats, scales, nullptr, centroids, segs, colors_in, n,
                          params, colors_out, stream);
}

// ---------------------------------------------------------------------------
// Probe fit for callers that cannot allocate device memory.
//
// sh_fit needs a dgsm_ctx, whose workspace is created with cudaMalloc.  Some
// callers cannot allocate: a real-time frame loop in which cudaMalloc and
// cudaFree would synchronise the device and stall the frame, or a host
// application that owns all device memory through its own pool and forbids
// allocations behind its back.  sh_fit_static runs the same two kernels with
// their per-block partial sums in a fixed array compiled into the library
// instead.
// ---------------------------------------------------------------------------
namespace {
constexpr int FIT_STATIC_BLOCKS = 256;  // partial-sum slots of the static scratch
constexpr int64_t FIT_STATIC_MAX_N = (int64_t)FIT_STATIC_BLOCKS * FIT_THREADS * 64;
constexpr int FIT_STATIC_STATUS = FIT_STATIC_BLOCKS * FIT_NV;  // index of the status word
constexpr int FIT_STATIC_DOUBLES = FIT_STATIC_STATUS + 32;
constexpr int FIT_STATIC_MAX_DEVICES = 64;
}  // namespace

// 256 x 72 partial sums + a status word: 147,712 bytes, held on every device
// that loads the library until the process exits.  Every call shares it.
static __device__ __align__(256) double dgsm_fit_scratch[FIT_STATIC_DOUBLES];

namespace {
std::mutex g_fit_scratch_mu;
double *g_fit_scratch_ptr[FIT_STATIC_MAX_DEVICES] = {};
unsigned long long g_fit_scratch_ctx[FIT_STATIC_MAX_DEVICES] = {};

// The id of the calling thread's current context (cuCtxGetId), or 0 when it
// cannot be read.  The two driver functions are looked up through the
// runtime, so the library links no driver library.  Call with
// g_fit_scratch_mu held.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        looked_up = true;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the static scratch on `dev` (which must be current).  In
// host code the symbol names a host-side stand-in, so the address is taken
// with cudaGetSymbolAddress and cached per device together with the id of
// the context it was taken in; it is taken again when the current context
// differs (after cudaDeviceReset, say) or its id cannot be read.
int fit_scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_fit_scratch_mu);
    const unsigned long long cid = current_context_id();
    if (!g_fit_scratch_ptr[dev] || cid == 0 || cid != g_fit_scratch_ctx[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, dgsm_fit_scratch) != cudaSuccess || !p)
            return DGSM_ERR_CUDA;
        g_fit_scratch_ptr[dev] = static_cast<double *>(p);
        // the runtime has made the device's context current by now
        g_fit_scratch_ctx[dev] = current_context_id();
    }
    *out = g_fit_scratch_ptr[dev];
    return DGSM_OK;
}
}  // namespace

extern "C" int sh_fit_static(const float *dirs, const float *rgb, const float *w, int64_t n,
                             double lambda, float *sh_out, double *sh64_out, int *status_out,
                             void *stream) {
    if (n < 1 || !dirs || !rgb || !w || !sh_out || !(lambda >= 0.0)) return DGSM_ERR_INVALID_ARG;
    if (n > FIT_STATIC_MAX_N) return DGSM_ERR_WORKSPACE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DGSM_ERR_CUDA;
    if (dev < 0 || dev >= FIT_STATIC_MAX_DEVICES) return DGSM_ERR_INVALID_ARG;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DGSM_ERR_CUDA;
    double *scratch = nullptr;
    int rc = fit_scratch_address(dev, &scratch);
    if (rc) return rc;
    int *status = reinterpret_cast<int *>(scratch + FIT_STATIC_STATUS);
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)std::min<int64_t>(
        std::min<int64_t>((n + FIT_THREADS - 1) / FIT_THREADS, (int64_t)sms), FIT_STATIC_BLOCKS);
    // an error left by earlier work of the caller's is reported, not cleared,
    // so that the launch check below sees this call's launches only
    if (cudaPeekAtLastError() != cudaSuccess) return DGSM_ERR_CUDA;
    // every partial slot the solve reads is rewritten below; only the status starts at zero
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return DGSM_ERR_CUDA;
    sh_fit_partial_kernel<<<nblocks, FIT_THREADS, 0, s>>>(dirs, rgb, w, n, scratch);
    sh_fit_solve_kernel<<<1, 128, 0, s>>>(scratch, nblocks, lambda, sh_out, sh64_out, status);
    if (cudaGetLastError() != cudaSuccess) return DGSM_ERR_CUDA;
    if (status_out &&
        cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return DGSM_ERR_CUDA;
    return DGSM_OK;
}
