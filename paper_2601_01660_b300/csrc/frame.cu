// frame.cu -- one shadowed and relit frame from host memory, and the
// alpha-weighted centroid that orients the relight normals.
//
// dgsm_frame_host strings the hot path together for callers whose Gaussians
// live in host memory: copy in, build the atlas from every Gaussian (Sec.
// 3.2), attenuate every Gaussian (Sec. 3.3), fit the probe (Sec. 3.4), relight
// the avatar range (Sec. 3.5) in place, copy the colours out.
#include <algorithm>

#include "dgsm_internal.cuh"
#include "motion.cuh"

namespace dgsm {
namespace {

__global__ void __launch_bounds__(CEN_THREADS) centroid_partial_kernel(
    const float *__restrict__ means, const float *__restrict__ w, int64_t n,
    double *__restrict__ partials) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w ? (double)w[i] : 1.0;
        a[0] += wi * means[3 * i];
        a[1] += wi * means[3 * i + 1];
        a[2] += wi * means[3 * i + 2];
        a[3] += wi;
    }
    __shared__ double red[CEN_THREADS / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < 4; ++c) {
        double x = a[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double x = 0.0;
        for (int q = 0; q < CEN_THREADS / 32; ++q) x += red[q][threadIdx.x];
        partials[4 * blockIdx.x + threadIdx.x] = x;
    }
}

__global__ void centroid_final_kernel(const double *__restrict__ partials, int nb,
                                      float *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < 4; ++c) a[c] += partials[4 * b + c];
    const double inv = a[3] > 0.0 ? 1.0 / a[3] : 0.0;
    out[0] = (float)(a[0] * inv);
    out[1] = (float)(a[1] * inv);
    out[2] = (float)(a[2] * inv);
}

// Per-object partial sums: blockIdx.y is the object, blockIdx.x strides
// over its Gaussians.
__global__ void __launch_bounds__(CEN_THREADS) segment_centroid_partial_kernel(
    const float *__restrict__ means, const float *__restrict__ w, const __grid_constant__ Segs segs,
    double *__restrict__ partials) {
    __shared__ double red[CEN_THREADS / 32][4];
    centroid_partial_block(
        w, segs, blockIdx.y, blockIdx.x, gridDim.x,
        [&](long long i) { return make_float3(means[3 * i], means[3 * i + 1], means[3 * i + 2]); }, partials,
        red);
}

// One warp per object.
__global__ void segment_centroid_final_kernel(const double *__restrict__ partials, int nb, int n_obj,
                                              float *__restrict__ out) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (o >= n_obj) return;
    centroid_final_warp(partials, nb, o, out);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_weighted_centroid(dgsm_ctx *ctx, const float *means, const float *weights,
                                      int64_t n, float *out, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || !out || (n > 0 && !means)) return fail(ctx, DGSM_ERR_INVALID_ARG, "centroid: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + CEN_THREADS - 1) / CEN_THREADS,
                                                               (int64_t)ctx->num_sms));
    void *part;
    int rc = ws_reserve(ctx, WS_CENTROID, sizeof(double) * 4 * nb, &part);
    if (rc) return rc;
    centroid_partial_kernel<<<nb, CEN_THREADS, 0, s>>>(means, weights, n, (double *)part);
    centroid_final_kernel<<<1, 32, 0, s>>>((const double *)part, nb, out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "centroid kernels");
}

extern "C" int dgsm_segment_centroids(dgsm_ctx *ctx, const float *means, const float *weights,
                                      int64_t n, const int64_t *seg, int32_t n_obj, float *out,
                                      void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    Segs segs;
    if (n < 0 || !out || (n > 0 && !means) || !make_segs(seg, n_obj, n, &segs))
        return fail(ctx, DGSM_ERR_INVALID_ARG,
                    "segment_centroids: bad arguments (need 1 <= n_obj <= 64, 0 = seg[0] <= ... <= seg[n_obj] = n)");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t longest = 0;
    for (int o = 0; o < n_obj; ++o) longest = std::max<int64_t>(longest, seg[o + 1] - seg[o]);
    const int bps = (int)std::max<int64_t>(
        1, std::min<int64_t>((longest + CEN_THREADS - 1) / CEN_THREADS,
                             std::max<int64_t>(1, 2 * (int64_t)ctx->num_sms / n_obj)));
    void *part;
    int rc = ws_reserve(ctx, WS_CENTROID, sizeof(double) * 4 * (size_t)bps * n_obj, &part);
    if (rc) return rc;
    segment_centroid_partial_kernel<<<dim3(bps, n_obj), CEN_THREADS, 0, s>>>(means, weights, segs,
                                                                           (double *)part);
    segment_centroid_final_kernel<<<(n_obj + 7) / 8, 256, 0, s>>>((const double *)part, bps, n_obj, out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "segment centroid kernels");
}

extern "C" int dgsm_frame_host(dgsm_ctx *ctx, const dgsm_frame_host_in *in,
                               const dgsm_params *params, const dgsm_relight_params *rparams,
                               float *colors_out, float *sh_out, void *stream) {
    DGSM_RANGE("dgsm_frame_host");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!in || !colors_out) return fail(ctx, DGSM_ERR_INVALID_ARG, "frame: null input or output");
    const int64_t n = in->n;
    if (n < 0 || in->relight_begin < 0 || in->relight_end < in->relight_begin || in->relight_end > n)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame: bad Gaussian count or relight range");
    if (n > 0 && (!in->means || !in->scales || !in->quats || !in->opac || !in->colors))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame: null Gaussian array");
    if (!in->lights || in->n_lights < 1 || in->n_lights > 64 || !in->radii || in->K < 1 || in->K > 256)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame: bad lights or radii");
    if (in->n_cube < 1 || !in->cube_dirs || !in->cube_rgb || !in->cube_w)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame: need cubemap samples");
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    const int L = in->n_lights, K = in->K, H = in->H, W = in->W;
    if (H < 1 || W < 1 || H > 4096 || W > 4096) return fail(ctx, DGSM_ERR_INVALID_ARG, "frame: bad H, W");
    const size_t esz = p.atlas_dtype == DGSM_F32 ? 4 : 2;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;

    // carve one device buffer
    const size_t sz_means = align256(12 * (size_t)n), sz_q = align256(16 * (size_t)n),
                 sz_op = align256(4 * (size_t)n), sz_l = align256(12 * (size_t)L),
                 sz_r = align256(4 * (size_t)K), sz_cube3 = align256(12 * (size_t)in->n_cube),
                 sz_cube1 = align256(4 * (size_t)in->n_cube),
                 sz_atlas = align256(esz * (size_t)L * K * H * W), sz_small = 256;
    const size_t total = 4 * sz_means + sz_q + sz_op + sz_l + sz_r + 2 * sz_cube3 + sz_cube1 +
                         sz_atlas + 2 * sz_small;
    void *base;
    int rc = ws_reserve(ctx, WS_FRAME, total, &base);
    if (rc) return rc;
    char *c = (char *)base;
    auto take = [&](size_t bytes) { char *r = c; c += bytes; return r; };
    float *d_means = (float *)take(sz_means), *d_scales = (float *)take(sz_means);
    float *d_colors = (float *)take(sz_means), *d_out = (float *)take(sz_means);
    float *d_quats = (float *)take(sz_q), *d_opac = (float *)take(sz_op);
    float *d_lights = (float *)take(sz_l), *d_radii = (float *)take(sz_r);
    float *d_cd = (float *)take(sz_cube3), *d_cr = (float *)take(sz_cube3);
    float *d_cw = (float *)take(sz_cube1);
    void *d_atlas = take(sz_atlas);
    float *d_sh = (float *)take(sz_small), *d_cen = (float *)take(sz_small);

    // Side stream: the colours and the cubemap go up, and the probe is fitted,
    // while the build runs on `stream`; the colours of the Gaussians that are
    // not relit come back while the avatar range is relit.
    if (!ctx->side) {
        e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
        for (int k = 0; e == cudaSuccess && k < 4; ++k)
            e = cudaEventCreateWithFlags(&ctx->fev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "frame: side stream");
    }
    cudaStream_t s2 = ctx->side;
    auto h2d = [&](void *dst, const void *src, size_t bytes, cudaStream_t st) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    e = cudaEventRecord(ctx->fev[0], s);  // the side stream starts after earlier work on `stream`
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ctx->fev[0], 0);
    // the build's inputs go up on both streams (two copy engines share the
    // host link); the build waits for the side stream's part
    if (e == cudaSuccess) e = h2d(d_means, in->means, 12 * (size_t)n, s);
    if (e == cudaSuccess) e = h2d(d_quats, in->quats, 16 * (size_t)n, s2);
    if (e == cudaSuccess) e = h2d(d_scales, in->scales, 12 * (size_t)n, s);
    if (e == cudaSuccess) e = h2d(d_opac, in->opac, 4 * (size_t)n, s2);
    if (e == cudaSuccess) e = h2d(d_lights, in->lights, 12 * (size_t)L, s);
    if (e == cudaSuccess) e = h2d(d_radii, in->radii, 4 * (size_t)K, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->fev[1], s2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->fev[1], 0);
    if (e == cudaSuccess) e = h2d(d_colors, in->colors, 12 * (size_t)n, s2);
    if (e == cudaSuccess) e = h2d(d_cd, in->cube_dirs, 12 * (size_t)in->n_cube, s2);
    if (e == cudaSuccess) e = h2d(d_cr, in->cube_rgb, 12 * (size_t)in->n_cube, s2);
    if (e == cudaSuccess) e = h2d(d_cw, in->cube_w, 4 * (size_t)in->n_cube, s2);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame: host to device copy");
    if ((rc = sh_fit(ctx, d_cd, d_cr, d_cw, in->n_cube, in->lambda, d_sh, nullptr, s2))) return rc;
    if ((e = cudaEventRecord(ctx->fev[1], s2)) != cudaSuccess) return cuda_fail(ctx, e, "frame: event");
    if ((rc = dgsm_build(ctx, d_means, d_scales, d_quats, d_opac, n, d_lights, L, H, W, d_radii, K,
                         &p, d_atlas, s)))
        return rc;
    if ((e = cudaStreamWaitEvent(s, ctx->fev[1], 0)) != cudaSuccess) return cuda_fail(ctx, e, "frame: wait");
    if ((rc = dgsm_attenuate(ctx, d_atlas, nullptr, p.atlas_dtype, L, H, W, d_radii, K, d_lights,
                             d_means, d_colors, n, nullptr, 1.0f, d_out, nullptr, s)))
        return rc;
    const int64_t a0 = in->relight_begin, a1 = in->relight_end, na = a1 - a0;
    // colours outside the relit range: back on the side stream, beside the relight
    if ((e = cudaEventRecord(ctx->fev[2], s)) != cudaSuccess) return cuda_fail(ctx, e, "frame: event");
    if ((e = cudaStreamWaitEvent(s2, ctx->fev[2], 0)) != cudaSuccess) return cuda_fail(ctx, e, "frame: wait");
    if (a0 > 0) e = cudaMemcpyAsync(colors_out, d_out, 12 * (size_t)a0, cudaMemcpyDeviceToHost, s2);
    if (e == cudaSuccess && a1 < n)
        e = cudaMemcpyAsync(colors_out + 3 * a1, d_out + 3 * a1, 12 * (size_t)(n - a1), cudaMemcpyDeviceToHost, s2);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame: device to host copy");
    if (na > 0) {
        if ((rc = dgsm_weighted_centroid(ctx, d_means + 3 * a0, d_opac + a0, na, d_cen, s))) return rc;
        if ((rc = sh_relight(ctx, d_sh, d_means + 3 * a0, d_quats + 4 * a0, d_scales + 3 * a0, nullptr,
                             d_cen, d_out + 3 * a0, na, rparams, d_out + 3 * a0, s)))
            return rc;
        e = cudaMemcpyAsync(colors_out + 3 * a0, d_out + 3 * a0, 12 * (size_t)na, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "frame: device to host copy");
    }
    if (sh_out) {
        e = cudaMemcpyAsync(sh_out, d_sh, 27 * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "frame: device to host copy");
    }
    if ((e = cudaEventRecord(ctx->fev[3], s2)) != cudaSuccess) return cuda_fail(ctx, e, "frame: event");
    if ((e = cudaStreamWaitEvent(s, ctx->fev[3], 0)) != cudaSuccess) return cuda_fail(ctx, e, "frame: wait");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame: synchronize");
    return dgsm_sync_status(ctx, stream);
}

// ---- pipelined host frames -------------------------------------------------
//
// dgsm_frame_host's work split so that frames overlap: a frame's inputs go
// up on the context's two copy-in streams (the two copy engines) as soon as it
// is submitted, its compute runs on the caller's stream after the frames
// submitted before it, and its colours come back on a copy-out stream.  While
// frame f computes, frame f + 1's inputs are copied in and frame f - 1's
// colours copied out.  Each of the two slots has its own device copies of the
// inputs, the atlas and the colours; the build's working buffers are the
// context's, which the caller's stream orders.

extern "C" int dgsm_frame_host_wait(dgsm_ctx *ctx, int slot) {
    if (!ctx || slot < 0 || slot > 1) return DGSM_ERR_INVALID_ARG;
    if (!ctx->fq_busy[slot]) return DGSM_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->fq_ev[slot][5]);
    ctx->fq_busy[slot] = false;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame wait: synchronize");
    const int st = ctx->fq_status[slot];
    return st == DGSM_OK ? DGSM_OK : fail(ctx, st, "frame wait: a kernel of the frame reported an error");
}

extern "C" int dgsm_frame_host_submit(dgsm_ctx *ctx, int slot, const dgsm_frame_host_in *in,
                                      const dgsm_params *params, const dgsm_relight_params *rparams,
                                      float *colors_out, float *sh_out, void *stream) {
    DGSM_RANGE("dgsm_frame_host_submit");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (slot < 0 || slot > 1) return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: slot must be 0 or 1");
    if (!in || !colors_out) return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: null input or output");
    const int64_t n = in->n;
    if (n < 0 || in->relight_begin < 0 || in->relight_end < in->relight_begin || in->relight_end > n)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: bad Gaussian count or relight range");
    if (n > 0 && (!in->means || !in->scales || !in->quats || !in->opac || !in->colors))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: null Gaussian array");
    if (!in->lights || in->n_lights < 1 || in->n_lights > 64 || !in->radii || in->K < 1 || in->K > 256)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: bad lights or radii");
    if (in->n_cube < 1 || !in->cube_dirs || !in->cube_rgb || !in->cube_w)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: need cubemap samples");
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    const int L = in->n_lights, K = in->K, H = in->H, W = in->W;
    if (H < 1 || W < 1 || H > 4096 || W > 4096) return fail(ctx, DGSM_ERR_INVALID_ARG, "frame submit: bad H, W");
    // the slot's previous frame still reads its buffers: finish it first
    int rc = dgsm_frame_host_wait(ctx, slot);
    if (rc) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (!ctx->fq_d2h) {
        for (int q = 0; e == cudaSuccess && q < 2; ++q)
            e = cudaStreamCreateWithFlags(&ctx->fq_h2d[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->fq_d2h, cudaStreamNonBlocking);
        for (int q = 0; q < 2; ++q)
            for (int k = 0; e == cudaSuccess && k < 6; ++k)
                e = cudaEventCreateWithFlags(&ctx->fq_ev[q][k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&ctx->fq_status, 2 * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "frame submit: streams");
    }
    const size_t esz = p.atlas_dtype == DGSM_F32 ? 4 : 2;
    const size_t sz_means = align256(12 * (size_t)n), sz_q = align256(16 * (size_t)n),
                 sz_op = align256(4 * (size_t)n), sz_l = align256(12 * (size_t)L),
                 sz_r = align256(4 * (size_t)K), sz_cube3 = align256(12 * (size_t)in->n_cube),
                 sz_cube1 = align256(4 * (size_t)in->n_cube),
                 sz_atlas = align256(esz * (size_t)L * K * H * W), sz_small = 256;
    const size_t total = 4 * sz_means + sz_q + sz_op + sz_l + sz_r + 2 * sz_cube3 + sz_cube1 +
                         sz_atlas + 2 * sz_small;
    void *base;
    if ((rc = ws_reserve(ctx, slot ? WS_FQ1 : WS_FQ0, total, &base))) return rc;
    char *c = (char *)base;
    auto take = [&](size_t bytes) { char *r = c; c += bytes; return r; };
    float *d_means = (float *)take(sz_means), *d_scales = (float *)take(sz_means);
    float *d_colors = (float *)take(sz_means), *d_out = (float *)take(sz_means);
    float *d_quats = (float *)take(sz_q), *d_opac = (float *)take(sz_op);
    float *d_lights = (float *)take(sz_l), *d_radii = (float *)take(sz_r);
    float *d_cd = (float *)take(sz_cube3), *d_cr = (float *)take(sz_cube3);
    float *d_cw = (float *)take(sz_cube1);
    void *d_atlas = take(sz_atlas);
    float *d_sh = (float *)take(sz_small), *d_cen = (float *)take(sz_small);

    const cudaStream_t s = (cudaStream_t)stream, ca = ctx->fq_h2d[0], cb = ctx->fq_h2d[1], cd = ctx->fq_d2h;
    cudaEvent_t *ev = ctx->fq_ev[slot];  // inputs a, inputs b, colours and cubemap, attenuated, relit, done
    auto h2d = [&](void *dst, const void *src, size_t bytes, cudaStream_t st) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    // copy in at once: nothing reads this slot's buffers any more
    e = h2d(d_means, in->means, 12 * (size_t)n, ca);
    if (e == cudaSuccess) e = h2d(d_quats, in->quats, 16 * (size_t)n, cb);
    if (e == cudaSuccess) e = h2d(d_scales, in->scales, 12 * (size_t)n, ca);
    if (e == cudaSuccess) e = h2d(d_opac, in->opac, 4 * (size_t)n, cb);
    if (e == cudaSuccess) e = h2d(d_lights, in->lights, 12 * (size_t)L, ca);
    if (e == cudaSuccess) e = h2d(d_radii, in->radii, 4 * (size_t)K, ca);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], ca);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], cb);
    if (e == cudaSuccess) e = h2d(d_colors, in->colors, 12 * (size_t)n, cb);
    if (e == cudaSuccess) e = h2d(d_cd, in->cube_dirs, 12 * (size_t)in->n_cube, cb);
    if (e == cudaSuccess) e = h2d(d_cr, in->cube_rgb, 12 * (size_t)in->n_cube, cb);
    if (e == cudaSuccess) e = h2d(d_cw, in->cube_w, 4 * (size_t)in->n_cube, cb);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], cb);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame submit: host to device copy");
    if ((rc = dgsm_build(ctx, d_means, d_scales, d_quats, d_opac, n, d_lights, L, H, W, d_radii, K, &p, d_atlas, s)))
        return rc;
    if ((e = cudaStreamWaitEvent(s, ev[2], 0)) != cudaSuccess) return cuda_fail(ctx, e, "frame submit: wait");
    if ((rc = sh_fit(ctx, d_cd, d_cr, d_cw, in->n_cube, in->lambda, d_sh, nullptr, s))) return rc;
    if ((rc = dgsm_attenuate(ctx, d_atlas, nullptr, p.atlas_dtype, L, H, W, d_radii, K, d_lights, d_means,
                             d_colors, n, nullptr, 1.0f, d_out, nullptr, s)))
        return rc;
    const int64_t a0 = in->relight_begin, a1 = in->relight_end, na = a1 - a0;
    // the colours outside the relit range go out while the range is relit
    e = cudaEventRecord(ev[3], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cd, ev[3], 0);
    if (e == cudaSuccess && a0 > 0) e = cudaMemcpyAsync(colors_out, d_out, 12 * (size_t)a0, cudaMemcpyDeviceToHost, cd);
    if (e == cudaSuccess && a1 < n)
        e = cudaMemcpyAsync(colors_out + 3 * a1, d_out + 3 * a1, 12 * (size_t)(n - a1), cudaMemcpyDeviceToHost, cd);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame submit: device to host copy");
    if (na > 0) {
        if ((rc = dgsm_weighted_centroid(ctx, d_means + 3 * a0, d_opac + a0, na, d_cen, s))) return rc;
        if ((rc = sh_relight(ctx, d_sh, d_means + 3 * a0, d_quats + 4 * a0, d_scales + 3 * a0, nullptr, d_cen,
                             d_out + 3 * a0, na, rparams, d_out + 3 * a0, s)))
            return rc;
    }
    // this frame's status word, then the word cleared for the next frame
    e = cudaMemcpyAsync(ctx->fq_status + slot, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cd, ev[4], 0);
    if (e == cudaSuccess && na > 0)
        e = cudaMemcpyAsync(colors_out + 3 * a0, d_out + 3 * a0, 12 * (size_t)na, cudaMemcpyDeviceToHost, cd);
    if (e == cudaSuccess && sh_out) e = cudaMemcpyAsync(sh_out, d_sh, 27 * sizeof(float), cudaMemcpyDeviceToHost, cd);
    if (e == cudaSuccess) e = cudaEventRecord(ev[5], cd);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame submit: device to host copy");
    ctx->fq_busy[slot] = true;
    return DGSM_OK;
}
