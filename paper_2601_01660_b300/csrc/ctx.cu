// ctx.cu -- context, errors, device status word and workspace of libdgsm.so.
#include <cstdio>
#include <cstring>
#include <new>

#include "dgsm_internal.cuh"

namespace dgsm {

int fail(dgsm_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(dgsm_ctx *ctx, cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return fail(ctx, DGSM_ERR_CUDA, buf);
}

bool make_segs(const int64_t *seg, int n_obj, int64_t n, Segs *out) {
    if (!seg || n_obj < 1 || n_obj > MAX_OBJECTS || seg[0] != 0 || seg[n_obj] != n) return false;
    for (int o = 0; o < n_obj; ++o)
        if (seg[o + 1] < seg[o]) return false;
    for (int o = 0; o <= MAX_OBJECTS; ++o) out->s[o] = o <= n_obj ? seg[o] : n;
    out->n = n_obj;
    return true;
}

int ws_reserve(dgsm_ctx *ctx, int slot, size_t bytes, void **out) {
    if (bytes == 0) bytes = 256;
    if (ctx->ws_cap[slot] < bytes) {
        if (ctx->frozen)
            return fail(ctx, DGSM_ERR_WORKSPACE,
                        "workspace would grow while a captured graph uses it: run the same calls "
                        "once before capturing");
        // grow by 25% headroom so that repeated builds of similar size do not reallocate
        size_t want = bytes + bytes / 4;
        if (ctx->ws[slot]) {
            cudaError_t e = cudaFree(ctx->ws[slot]);  // synchronises the device
            ctx->ws[slot] = nullptr;
            ctx->ws_cap[slot] = 0;
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(workspace)");
        }
        cudaError_t e = cudaMalloc(&ctx->ws[slot], want);
        if (e != cudaSuccess) {
            ctx->ws[slot] = nullptr;
            return cuda_fail(ctx, e, "cudaMalloc(workspace)");
        }
        ctx->ws_cap[slot] = want;
    }
    *out = ctx->ws[slot];
    return DGSM_OK;
}

}  // namespace dgsm

using namespace dgsm;

extern "C" void dgsm_default_params(dgsm_params *p) {
    if (!p) return;
    p->kappa = 1.0f;
    p->eps_cull = 1e-7f;
    p->tile = 8;
    p->chunk = 128;
    p->atlas_dtype = DGSM_F32;
    p->max_pairs = 0;
    p->beta_mode = 2;
    p->atlas_map = 0;
}

extern "C" void dgsm_default_relight_params(dgsm_relight_params *p) {
    if (!p) return;
    p->q = 1.0f;
    p->gamma = 1.0f;
    p->t_max = 10.0f;
    p->eps = 1e-8f;
    p->n_theta = 32;
    p->n_phi = 64;
}

extern "C" int dgsm_create(int device, dgsm_ctx **out) {
    if (!out) return DGSM_ERR_INVALID_ARG;
    *out = nullptr;
    dgsm_ctx *ctx = new (std::nothrow) dgsm_ctx();
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stats, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 16 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        dgsm_destroy(ctx);
        return DGSM_ERR_CUDA;
    }
    *out = ctx;
    return DGSM_OK;
}

extern "C" void dgsm_destroy(dgsm_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (int s = 0; s < WS_NSLOTS; ++s)
        if (ctx->ws[s]) cudaFree(ctx->ws[s]);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_stats) cudaFree(ctx->d_stats);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    for (int b = 0; b < dgsm_ctx::PROF_RING; ++b)
        for (int k = 0; k < 3; ++k)
            if (ctx->prof_ev[b][k]) cudaEventDestroy(ctx->prof_ev[b][k]);
    for (int k = 0; k < 4; ++k)
        if (ctx->fev[k]) cudaEventDestroy(ctx->fev[k]);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (int q = 0; q < 2; ++q) {
        for (int k = 0; k < 6; ++k)
            if (ctx->fq_ev[q][k]) cudaEventDestroy(ctx->fq_ev[q][k]);
        if (ctx->fq_h2d[q]) cudaStreamDestroy(ctx->fq_h2d[q]);
    }
    if (ctx->fq_d2h) cudaStreamDestroy(ctx->fq_d2h);
    if (ctx->fq_status) cudaFreeHost(ctx->fq_status);
    delete ctx;
}

extern "C" const char *dgsm_last_error(const dgsm_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" const char *dgsm_status_string(int status) {
    switch (status) {
        case DGSM_OK: return "ok";
        case DGSM_ERR_INVALID_ARG: return "invalid argument";
        case DGSM_ERR_CUDA: return "CUDA error";
        case DGSM_ERR_WORKSPACE: return "workspace or output capacity too small";
        case DGSM_ERR_TIMEOUT: return "device-side wait timed out";
        case DGSM_ERR_NONFINITE_INPUT: return "non-finite or non-positive Gaussian input";
        case DGSM_ERR_NOT_SPD: return "normal equations not positive definite";
        default: return "unknown status";
    }
}

extern "C" int dgsm_sync_status(dgsm_ctx *ctx, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dgsm_sync_status");
    int code = *(int *)ctx->h_pinned;
    if (code != DGSM_OK) return fail(ctx, code, std::string("device status: ") + dgsm_status_string(code));
    return DGSM_OK;
}

extern "C" int dgsm_set_profiling(dgsm_ctx *ctx, int enable) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (enable && !ctx->prof_ev[0][0]) {
        for (int b = 0; b < dgsm_ctx::PROF_RING; ++b)
            for (int k = 0; k < 3; ++k) {
                e = cudaEventCreate(&ctx->prof_ev[b][k]);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
            }
    }
    ctx->prof = enable != 0;
    ctx->prof_count = 0;
    return DGSM_OK;
}

extern "C" int dgsm_profile_collect(dgsm_ctx *ctx, double *ms_out, int max_builds, int *n_out) {
    if (!ctx || !n_out || max_builds < 0 || (max_builds > 0 && !ms_out)) return DGSM_ERR_INVALID_ARG;
    const int n = ctx->prof_count < dgsm_ctx::PROF_RING ? ctx->prof_count : dgsm_ctx::PROF_RING;
    int w = 0;
    for (int b = 0; b < n && w < max_builds; ++b, ++w) {
        float a = 0.f, c = 0.f;
        cudaError_t e = cudaEventSynchronize(ctx->prof_ev[b][2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ctx->prof_ev[b][0], ctx->prof_ev[b][1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&c, ctx->prof_ev[b][1], ctx->prof_ev[b][2]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dgsm_profile_collect");
        ms_out[2 * w] = a;
        ms_out[2 * w + 1] = c;
    }
    *n_out = w;
    ctx->prof_count = 0;
    return DGSM_OK;
}
