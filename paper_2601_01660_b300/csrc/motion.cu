// motion.cu -- rigid motion of whole objects (avatars) made of Gaussians.
//
// A rigid pose (rotation q_o, translation t) moves a Gaussian to mean
// R(q_o) mu + t and rotation q_o * q (Hamilton product), so that its
// covariance becomes R(q_o) Sigma R(q_o)^T with the scales unchanged.  The
// moved Gaussians are what the per-frame dynamic atlas is built from
// (Sec. 3.2) and what the receivers of a frame are (Sec. 3.3).
#include <algorithm>

#include "dgsm_internal.cuh"
#include "motion.cuh"

namespace dgsm {
namespace {

constexpr int RT_THREADS = 256;

__global__ void __launch_bounds__(RT_THREADS) rigid_transform_kernel(
    const float *__restrict__ means, const float *__restrict__ quats, int64_t n,
    const __grid_constant__ Segs segs, const float *__restrict__ poses, float *__restrict__ means_out,
    float *__restrict__ quats_out) {
    // per object: unit rotation quaternion (w,x,y,z), translation, row-major R
    __shared__ float P[MAX_OBJECTS][16];
    for (int o = threadIdx.x; o < segs.n; o += blockDim.x) pose_matrix(poses + 8 * o, P[o]);
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const float *r = P[segs.n == 1 ? 0 : seg_find(segs, g)];
        const float3 m = pose_point(r, means[3 * g], means[3 * g + 1], means[3 * g + 2]);
        means_out[3 * g] = m.x;
        means_out[3 * g + 1] = m.y;
        means_out[3 * g + 2] = m.z;
        reinterpret_cast<float4 *>(quats_out)[g] = pose_quat(r, reinterpret_cast<const float4 *>(quats)[g]);
    }
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_rigid_transform(dgsm_ctx *ctx, const float *means, const float *quats,
                                    int64_t n, const int64_t *seg, int32_t n_obj,
                                    const float *poses, float *means_out, float *quats_out,
                                    void *stream) {
    DGSM_RANGE("dgsm_rigid_transform");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "rigid_transform: n < 0");
    Segs segs;
    if (!make_segs(seg, n_obj, n, &segs))
        return fail(ctx, DGSM_ERR_INVALID_ARG,
                    "rigid_transform: need 1 <= n_obj <= 64 and 0 = seg[0] <= ... <= seg[n_obj] = n");
    if (!poses) return fail(ctx, DGSM_ERR_INVALID_ARG, "rigid_transform: null poses");
    if (n > 0 && (!means || !quats || !means_out || !quats_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "rigid_transform: null Gaussian array");
    if (((uintptr_t)quats | (uintptr_t)quats_out) & 15)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "rigid_transform: quaternion arrays must be 16-byte aligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    void *d_poses;
    int rc = ws_reserve(ctx, WS_POSES, sizeof(float) * 8 * MAX_OBJECTS, &d_poses);
    if (rc) return rc;
    // host (pinned, for graph capture) or device poses: the copy reads them
    // when it runs on the stream
    e = cudaMemcpyAsync(d_poses, poses, sizeof(float) * 8 * (size_t)n_obj, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rigid_transform: pose copy");
    if (n == 0) return DGSM_OK;
    const int grid = (int)std::min<int64_t>((n + RT_THREADS - 1) / RT_THREADS, (int64_t)ctx->num_sms * 8);
    rigid_transform_kernel<<<grid, RT_THREADS, 0, s>>>(means, quats, n, segs, (const float *)d_poses,
                                                       means_out, quats_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "rigid_transform_kernel");
}
