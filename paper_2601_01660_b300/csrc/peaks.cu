// peaks.cu -- measured single-precision ALU peaks of this GPU: the roofline
// denominators of the build's tile kernel, which is bound by FP32 and
// special-function (MUFU) issue rather than by memory.
//
// Each kernel keeps every SM full (2048 threads) with eight independent
// dependency chains per thread, so throughput, not latency, is measured:
//   fp32_kernel   chains of FFMA (one FP32 operation per lane and instruction)
//   mufu_kernel   chains of ex2.approx, rcp.approx or rsqrt.approx (the rcp
//                 chain adds 0.5 between steps, an FMA-pipe add, so that no
//                 two reciprocals cancel)
// The result is stored only under a condition no input meets, so nothing is
// optimised away, and nothing is written in practice.
#include <algorithm>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_BLOCKS_PER_SM = 8;
constexpr int PK_CHAINS = 8;
constexpr int PK_UNROLL = 16;

__global__ void __launch_bounds__(PK_THREADS) fp32_kernel(float *sink, int iters, float a, float b) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.2345e30f) sink[0] = s;
}

template <int OP>
__device__ __forceinline__ float mufu(float x) {
    float y;
    if (OP == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    else if (OP == 1) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x + 0.5f));
    else asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(PK_THREADS) mufu_kernel(float *sink, int iters) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 0.5f + (float)((threadIdx.x + c) & 7) * 0.0625f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = mufu<OP>(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    if (s == -1.2345e30f) sink[0] = s;
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

// out[0]: FP32 FFMA lane operations per second; out[1..3]: ex2.approx,
// rcp.approx, rsqrt.approx lane operations per second.  Best of three timed
// launches each, after one untimed launch.  Blocks until done.
extern "C" int dgsm_measure_alu_peaks(dgsm_ctx *ctx, double *out, void *stream) {
    if (!ctx || !out) return DGSM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    float *sink = nullptr;
    int rc = ws_reserve(ctx, WS_SCAN_TMP, 256, (void **)&sink);
    if (rc != DGSM_OK) return rc;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    const int grid = ctx->num_sms * PK_BLOCKS_PER_SM;
    const double per_iter = (double)grid * PK_THREADS * PK_UNROLL * PK_CHAINS;
    // about 25 ms per FP32 launch and 40 ms per MUFU launch at the B300's nominal rates
    const int it_fp32 = 8192, it_mufu = 1536;
    auto time_one = [&](int which) -> double {
        double best = 1e30;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(ev[0], s);
            if (e != cudaSuccess) break;
            switch (which) {
                case 0: fp32_kernel<<<grid, PK_THREADS, 0, s>>>(sink, it_fp32, 0.999f, 1e-3f); break;
                case 1: mufu_kernel<0><<<grid, PK_THREADS, 0, s>>>(sink, it_mufu); break;
                case 2: mufu_kernel<1><<<grid, PK_THREADS, 0, s>>>(sink, it_mufu); break;
                default: mufu_kernel<2><<<grid, PK_THREADS, 0, s>>>(sink, it_mufu); break;
            }
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e == cudaSuccess && rep > 0 && ms > 0.f) best = std::min(best, (double)ms);
        }
        return best;
    };
    for (int which = 0; which < 4 && e == cudaSuccess; ++which) {
        const double ms = time_one(which);
        const double ops = per_iter * (which == 0 ? it_fp32 : it_mufu);
        out[which] = ops / (ms * 1e-3);
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "dgsm_measure_alu_peaks");
}
