// motion.cu -- rigid motion of whole objects (avatars) made of Gaussians.
//
// A rigid pose (rotation q_o, translation t) moves a Gaussian to mean
// R(q_o) mu + t and rotation q_o * q (Hamilton product), so that its
// covariance becomes R(q_o) Sigma R(q_o)^T with the scales unchanged.  The
// moved Gaussians are what the per-frame dynamic atlas is built from
// (Sec. 3.2) and what the receivers of a frame are (Sec. 3.3).
#include <algorithm>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int RT_THREADS = 256;

__global__ void __launch_bounds__(RT_THREADS) rigid_transform_kernel(
    const float *__restrict__ means, const float *__restrict__ quats, int64_t n,
    const __grid_constant__ Segs segs, const float *__restrict__ poses, float *__restrict__ means_out,
    float *__restrict__ quats_out) {
    // per object: unit rotation quaternion (w,x,y,z), translation, row-major R
    __shared__ float P[MAX_OBJECTS][16];
    for (int o = threadIdx.x; o < segs.n; o += blockDim.x) {
        float w = poses[8 * o], x = poses[8 * o + 1], y = poses[8 * o + 2], z = poses[8 * o + 3];
        const float inv = rsqrtf(w * w + x * x + y * y + z * z);
        w *= inv; x *= inv; y *= inv; z *= inv;
        float *r = P[o];
        r[0] = w; r[1] = x; r[2] = y; r[3] = z;
        r[4] = poses[8 * o + 4]; r[5] = poses[8 * o + 5]; r[6] = poses[8 * o + 6];
        r[7] = 1.f - 2.f * (y * y + z * z); r[8] = 2.f * (x * y - w * z); r[9] = 2.f * (x * z + w * y);
        r[10] = 2.f * (x * y + w * z); r[11] = 1.f - 2.f * (x * x + z * z); r[12] = 2.f * (y * z - w * x);
        r[13] = 2.f * (x * z - w * y); r[14] = 2.f * (y * z + w * x); r[15] = 1.f - 2.f * (x * x + y * y);
    }
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const float *r = P[segs.n == 1 ? 0 : seg_find(segs, g)];
        const float mx = means[3 * g], my = means[3 * g + 1], mz = means[3 * g + 2];
        means_out[3 * g] = r[7] * mx + r[8] * my + r[9] * mz + r[4];
        means_out[3 * g + 1] = r[10] * mx + r[11] * my + r[12] * mz + r[5];
        means_out[3 * g + 2] = r[13] * mx + r[14] * my + r[15] * mz + r[6];
        const float4 q = reinterpret_cast<const float4 *>(quats)[g];  // (w, x, y, z)
        const float w1 = r[0], x1 = r[1], y1 = r[2], z1 = r[3];
        float4 o;
        o.x = w1 * q.x - x1 * q.y - y1 * q.z - z1 * q.w;
        o.y = w1 * q.y + x1 * q.x + y1 * q.w - z1 * q.z;
        o.z = w1 * q.z - x1 * q.w + y1 * q.x + z1 * q.y;
        o.w = w1 * q.w + x1 * q.z - y1 * q.y + z1 * q.x;
        reinterpret_cast<float4 *>(quats_out)[g] = o;
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
