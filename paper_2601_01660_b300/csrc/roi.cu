// roi.cu -- the box of a receiver-driven region of interest (Sec. 3.2).
//
// c = the alpha-weighted centroid (x, y) of an avatar's Gaussians and the
// height range of their centres, padded; dgsm_build_roi (build.cu) takes the
// box and restricts the build to the texels and shells its receivers read.
#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int BOX_THREADS = 1024;

// One block: per-thread float sums over a strided share of the avatar, then
// the 1024 partial sums combined in double.
__global__ void __launch_bounds__(BOX_THREADS) roi_box_kernel(const float *__restrict__ means,
                                                              const float *__restrict__ opac, int64_t n,
                                                              float R, float z_margin, float *__restrict__ box) {
    __shared__ double sw[BOX_THREADS / 32], sx[BOX_THREADS / 32], sy[BOX_THREADS / 32];
    __shared__ float szl[BOX_THREADS / 32], szh[BOX_THREADS / 32];
    float w = 0.0f, ax = 0.0f, ay = 0.0f;
    float zl = INFINITY, zh = -INFINITY;
    for (int64_t g = threadIdx.x; g < n; g += BOX_THREADS) {
        const float a = __ldg(opac + g);
        w += a;
        ax = fmaf(a, __ldg(means + 3 * g), ax);
        ay = fmaf(a, __ldg(means + 3 * g + 1), ay);
        const float z = __ldg(means + 3 * g + 2);
        zl = fminf(zl, z);
        zh = fmaxf(zh, z);
    }
    double dw = w, dx = ax, dy = ay;
    for (int o = 16; o > 0; o >>= 1) {
        dw += __shfl_down_sync(0xffffffffu, dw, o);
        dx += __shfl_down_sync(0xffffffffu, dx, o);
        dy += __shfl_down_sync(0xffffffffu, dy, o);
        zl = fminf(zl, __shfl_down_sync(0xffffffffu, zl, o));
        zh = fmaxf(zh, __shfl_down_sync(0xffffffffu, zh, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sw[warp] = dw;
        sx[warp] = dx;
        sy[warp] = dy;
        szl[warp] = zl;
        szh[warp] = zh;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double W = 0.0, X = 0.0, Y = 0.0;
        float lo = INFINITY, hi = -INFINITY;
        for (int k = 0; k < BOX_THREADS / 32; ++k) {
            W += sw[k];
            X += sx[k];
            Y += sy[k];
            lo = fminf(lo, szl[k]);
            hi = fmaxf(hi, szh[k]);
        }
        const bool ok = W > 0.0;
        box[0] = ok ? (float)(X / W) : 0.0f;
        box[1] = ok ? (float)(Y / W) : 0.0f;
        box[2] = ok ? R : -1.0f;  // no weight: an empty box
        box[3] = lo - z_margin;
        box[4] = hi + z_margin;
    }
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_roi_box(dgsm_ctx *ctx, const float *avatar_means, const float *avatar_opac, int64_t n,
                            float R, float z_margin, float *box_out, void *stream) {
    DGSM_RANGE("dgsm_roi_box");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 1 || !avatar_means || !avatar_opac || !box_out)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "roi box: need n >= 1 and device arrays");
    if (!(R >= 0.0f) || !(z_margin >= 0.0f)) return fail(ctx, DGSM_ERR_INVALID_ARG, "roi box: R, z_margin >= 0");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    roi_box_kernel<<<1, BOX_THREADS, 0, (cudaStream_t)stream>>>(avatar_means, avatar_opac, n, R, z_margin,
                                                                box_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "roi_box_kernel");
}
