// motion.cuh -- rigid motion of whole objects and their alpha-weighted
// centroids (the reference points of the relight normals, Sec. 3.5) as
// device functions, shared by the standalone kernels (motion.cu, frame.cu)
// and the persistent frame kernel, so that both compute the same floats.
#pragma once

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

// Pose (qw, qx, qy, qz, tx, ty, tz, -) -> r[16]: the unit quaternion,
// the translation, then R(q) row-major.
__device__ __forceinline__ void pose_matrix(const float *pose, float *r) {
    float w = pose[0], x = pose[1], y = pose[2], z = pose[3];
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    r[0] = w; r[1] = x; r[2] = y; r[3] = z;
    r[4] = pose[4]; r[5] = pose[5]; r[6] = pose[6];
    r[7] = 1.f - 2.f * (y * y + z * z); r[8] = 2.f * (x * y - w * z); r[9] = 2.f * (x * z + w * y);
    r[10] = 2.f * (x * y + w * z); r[11] = 1.f - 2.f * (x * x + z * z); r[12] = 2.f * (y * z - w * x);
    r[13] = 2.f * (x * z - w * y); r[14] = 2.f * (y * z + w * x); r[15] = 1.f - 2.f * (x * x + y * y);
}

// The moved mean R m + t.
__device__ __forceinline__ float3 pose_point(const float *r, float mx, float my, float mz) {
    return make_float3(r[7] * mx + r[8] * my + r[9] * mz + r[4], r[10] * mx + r[11] * my + r[12] * mz + r[5],
                       r[13] * mx + r[14] * my + r[15] * mz + r[6]);
}

// The moved rotation q_pose * q (Hamilton product), q = (w, x, y, z) stored
// as a float4 (x = w, y = x, z = y, w = z).
__device__ __forceinline__ float4 pose_quat(const float *r, float4 q) {
    const float w1 = r[0], x1 = r[1], y1 = r[2], z1 = r[3];
    float4 o;
    o.x = w1 * q.x - x1 * q.y - y1 * q.z - z1 * q.w;
    o.y = w1 * q.y + x1 * q.x + y1 * q.w - z1 * q.z;
    o.z = w1 * q.z - x1 * q.w + y1 * q.x + z1 * q.y;
    o.w = w1 * q.w + x1 * q.z - y1 * q.y + z1 * q.x;
    return o;
}

constexpr int CEN_THREADS = 256;

// Partial FP64 sums (sum w x, sum w y, sum w z, sum w) of object o over its
// Gaussians i = s[o] + part * 256 + tid, stepping by nparts * 256, reduced
// over the block in a fixed order into partials[4 (o nparts + part) + c].
// point(i) gives the Gaussian's (moved) mean.  256 threads; all call it.
template <typename PointF>
__device__ __forceinline__ void centroid_partial_block(const float *__restrict__ w, const Segs &segs, int o,
                                                       int part, int nparts, PointF point,
                                                       double *__restrict__ partials, double (*red)[4]) {
    const long long b = segs.s[o], e = segs.s[o + 1];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = b + (long long)part * CEN_THREADS + threadIdx.x; i < e;
         i += (long long)nparts * CEN_THREADS) {
        const double wi = w ? (double)w[i] : 1.0;
        const float3 m = point(i);
        a[0] += wi * m.x;
        a[1] += wi * m.y;
        a[2] += wi * m.z;
        a[3] += wi;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < 4; ++c) {
        double x = a[c];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double x = 0.0;
        for (int q = 0; q < CEN_THREADS / 32; ++q) x += red[q][threadIdx.x];
        partials[4 * ((int64_t)o * nparts + part) + threadIdx.x] = x;
    }
    __syncthreads();  // red is reused by the next call
}

// One warp: the centroid of object o from its nparts partial sums (summed
// lane-strided, then across the warp), 0 for a weightless object.
__device__ __forceinline__ void centroid_final_warp(const double *partials, int nparts, int o, float *out) {
    const int lane = threadIdx.x & 31;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = lane; b < nparts; b += 32)
        for (int c = 0; c < 4; ++c) a[c] += __ldcg(partials + 4 * ((int64_t)o * nparts + b) + c);
    for (int c = 0; c < 4; ++c)
        for (int off = 16; off > 0; off >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], off);
    if (lane == 0) {
        const double inv = a[3] > 0.0 ? 1.0 / a[3] : 0.0;
        out[3 * o] = (float)(a[0] * inv);
        out[3 * o + 1] = (float)(a[1] * inv);
        out[3 * o + 2] = (float)(a[2] * inv);
    }
}

}  // namespace
}  // namespace dgsm
