// runtime.cu -- frame-loop mechanics: CUDA-graph capture of library calls,
// and a measured choice of the build's tile and chunk.
//
// A frame of the moving-avatar workload (rigid motion, dynamic-atlas build,
// attenuation against static x dynamic atlases, per-avatar relight) is a
// few dozen kernel launches.  Captured once into a CUDA graph and replayed,
// it costs one launch per frame and no host work; the build's capacity mode
// (dgsm_params.max_pairs) keeps it free of host synchronisation.
#include <algorithm>
#include <vector>

#include "dgsm_internal.cuh"

struct dgsm_graph {
    dgsm_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace dgsm;

extern "C" int dgsm_graph_begin(dgsm_ctx *ctx, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!stream)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "graph capture needs a created stream, not the legacy default stream");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    e = cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    ++ctx->frozen;
    return DGSM_OK;
}

extern "C" int dgsm_graph_end(dgsm_ctx *ctx, void *stream, dgsm_graph **out) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!out) return fail(ctx, DGSM_ERR_INVALID_ARG, "graph_end: null output");
    *out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &g);
    if (e != cudaSuccess || !g) {
        --ctx->frozen;
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, e != cudaSuccess ? e : cudaErrorStreamCaptureInvalidated, "cudaStreamEndCapture");
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        --ctx->frozen;
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    dgsm_graph *G = new dgsm_graph;
    G->ctx = ctx;
    G->graph = g;
    G->exec = x;
    *out = G;
    return DGSM_OK;
}

extern "C" int dgsm_graph_launch(dgsm_graph *g, void *stream) {
    if (!g) return DGSM_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? DGSM_OK : cuda_fail(g->ctx, e, "cudaGraphLaunch");
}

extern "C" int dgsm_graph_node_count(dgsm_graph *g, int64_t *n_out) {
    if (!g || !n_out) return DGSM_ERR_INVALID_ARG;
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(g->graph, nullptr, &n);
    if (e != cudaSuccess) return cuda_fail(g->ctx, e, "cudaGraphGetNodes");
    *n_out = (int64_t)n;
    return DGSM_OK;
}

extern "C" void dgsm_graph_destroy(dgsm_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->ctx && g->ctx->frozen > 0) --g->ctx->frozen;
    delete g;
}

extern "C" int dgsm_autotune_build(dgsm_ctx *ctx, const float *means, const float *scales,
                                   const float *quats, const float *opac, int64_t n,
                                   const float *lights, int32_t L, int32_t H, int32_t W,
                                   const float *radii, int32_t K, const dgsm_params *base,
                                   const int32_t *tiles, int32_t n_tiles, const int32_t *chunks,
                                   int32_t n_chunks, int32_t reps, void *atlas,
                                   dgsm_params *best_out, float *ms_out, void *stream) {
    DGSM_RANGE("dgsm_autotune_build");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!tiles || !chunks || n_tiles < 1 || n_chunks < 1 || reps < 1 || !best_out)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "autotune: need candidates, reps >= 1 and an output");
    dgsm_params p0;
    if (base) p0 = *base; else dgsm_default_params(&p0);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev0, ev1;
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ev1)) != cudaSuccess) {
        cudaEventDestroy(ev0);
        return cuda_fail(ctx, e, "cudaEventCreate");
    }
    float best_ms = -1.0f;
    int rc = DGSM_OK;
    std::vector<float> t(reps);
    for (int a = 0; a < n_tiles && rc == DGSM_OK; ++a) {
        for (int b = 0; b < n_chunks && rc == DGSM_OK; ++b) {
            dgsm_params p = p0;
            p.tile = tiles[a];
            p.chunk = chunks[b];
            float med = -1.0f;
            // a candidate the build rejects (tile or shared memory) is skipped
            int r = dgsm_build(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, &p, atlas, s);
            if (r == DGSM_OK) {
                for (int k = 0; k < reps && r == DGSM_OK; ++k) {
                    cudaEventRecord(ev0, s);
                    r = dgsm_build(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, &p, atlas, s);
                    cudaEventRecord(ev1, s);
                    if (r == DGSM_OK && (e = cudaEventSynchronize(ev1)) == cudaSuccess)
                        e = cudaEventElapsedTime(&t[k], ev0, ev1);
                    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "autotune timing");
                }
                if (r == DGSM_OK && rc == DGSM_OK) {
                    std::sort(t.begin(), t.end());
                    med = t[reps / 2];
                }
            }
            if (r != DGSM_OK && r != DGSM_ERR_INVALID_ARG) rc = r;  // a real failure
            if (ms_out) ms_out[a * n_chunks + b] = med;
            if (med >= 0.0f && (best_ms < 0.0f || med < best_ms)) {
                best_ms = med;
                *best_out = p;
            }
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (rc != DGSM_OK) return rc;
    if (best_ms < 0.0f) return fail(ctx, DGSM_ERR_INVALID_ARG, "autotune: no candidate ran");
    return DGSM_OK;
}
