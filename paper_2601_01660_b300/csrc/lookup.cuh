// lookup.cuh -- the trilinear atlas lookup of Sec. 3.3 (bilinear between
// texel centres with clamp-to-edge, linear between the bracketing shells),
// shared by the attenuation kernels and the persistent frame kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

template <typename T>
__device__ __forceinline__ float load_T(const T *p);
template <>
__device__ __forceinline__ float load_T<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_T<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float load_T<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}

// An atlas value read through L2 only (an atlas written earlier by the same
// kernel, which the read-only cache path may not see).
__device__ __forceinline__ float load_cg(const float *p) { return __ldcg(p); }

// Trilinear lookup in one light's atlas A [K][H][W] (at most 2^32 voxels, so
// 32-bit offsets); inw[k] = 1 / (radii[k+1] - radii[k]).  CG: read the taps
// with load_cg (float atlases only).
template <typename T, bool CG = false>
__device__ __forceinline__ float lookup(const T *__restrict__ A, int H, int W, int K,
                                        const SampleIndex &s, const float *rs, const float *inw) {
    // rows clamped to the point's face (the whole atlas for the octahedral map)
    const int j0 = min(max(s.bj, 0), W - 1), j1 = min(max(s.bj + 1, 0), W - 1);
    const int rlo = s.r0, rhi = s.r0 + s.hf - 1;
    const int i0 = min(max(s.bi, rlo), rhi), i1 = min(max(s.bi + 1, rlo), rhi);
    int k0, k1;
    float wt;
    if (s.k < 0) { k0 = k1 = 0; wt = 0.0f; }
    else if (s.k >= K - 1) { k0 = k1 = K - 1; wt = 0.0f; }
    else { k0 = s.k; k1 = s.k + 1; wt = (s.t - rs[k0]) * inw[k0]; }
    const uint32_t plane = (uint32_t)H * (uint32_t)W;
    const uint32_t o00 = (uint32_t)i0 * W + j0, o01 = (uint32_t)i0 * W + j1;
    const uint32_t o10 = (uint32_t)i1 * W + j0, o11 = (uint32_t)i1 * W + j1;
    const float fx = s.fx, fy = s.fy;
    auto ld = [](const T *p) {
        if constexpr (CG) return load_cg(p);
        else return load_T<T>(p);
    };
    const T *P0 = A + (uint32_t)k0 * plane;
    float b0 = (1.0f - fy) * ((1.0f - fx) * ld(P0 + o00) + fx * ld(P0 + o01)) +
               fy * ((1.0f - fx) * ld(P0 + o10) + fx * ld(P0 + o11));
    if (k1 == k0) return b0;
    const T *P1 = A + (uint32_t)k1 * plane;
    float b1 = (1.0f - fy) * ((1.0f - fx) * ld(P1 + o00) + fx * ld(P1 + o01)) +
               fy * ((1.0f - fx) * ld(P1 + o10) + fx * ld(P1 + o11));
    return (1.0f - wt) * b0 + wt * b1;
}

}  // namespace
}  // namespace dgsm
