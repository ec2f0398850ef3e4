// relight.cuh -- the real SH basis of the probe fit (Sec. 3.4) and the
// pieces of the per-Gaussian radiance transfer (Sec. 3.5, Eqs. 8-10), shared
// by sh.cu's kernels and the persistent frame kernel.
#pragma once

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

// Real SH basis to degree 2, index l^2 + l + m, no Condon-Shortley phase.
// Normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for
// m != 0, with the Cartesian forms of the associated Legendre factors.
constexpr double SH_C0 = 0.28209479177387814;   // 1/2 sqrt(1/pi)
constexpr double SH_C1 = 0.48860251190291992;   // sqrt(3/(4 pi))
constexpr double SH_C2 = 1.09254843059207907;   // 1/2 sqrt(15/pi)
constexpr double SH_C20 = 0.31539156525252005;  // 1/4 sqrt(5/pi)
constexpr double SH_C22 = 0.54627421529603959;  // 1/4 sqrt(15/pi)

template <typename F>
__device__ __forceinline__ void sh9(F x, F y, F z, F *Y) {
    Y[0] = F(SH_C0);
    Y[1] = F(SH_C1) * y;
    Y[2] = F(SH_C1) * z;
    Y[3] = F(SH_C1) * x;
    Y[4] = F(SH_C2) * x * y;
    Y[5] = F(SH_C2) * y * z;
    Y[6] = F(SH_C20) * (F(3) * z * z - F(1));
    Y[7] = F(SH_C2) * x * z;
    Y[8] = F(SH_C22) * (x * x - y * y);
}

// Entries j in [j0, j1) of the transfer's direction table (block-strided):
// tab[2 (j - j0)] = (omega_j, w_j), tab[2 (j - j0) + 1] = (w_j L(omega_j), 0),
// lat-long cell centres theta = (i + 1/2) pi / nth, phi = (p + 1/2) 2 pi / nph,
// w = sin(theta); L the probe's radiance from its 3 x 9 coefficients shs.
__device__ __forceinline__ void relight_table_fill(const float *shs, int j0, int j1, int nth, int nph,
                                                   float4 *tab) {
    for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
        const int it = j / nph, ip = j - it * nph;
        float st, ct, sp, cp;
        sincospif((it + 0.5f) / nth, &st, &ct);
        sincospif(2.0f * (ip + 0.5f) / nph, &sp, &cp);
        const float ox = st * cp, oy = st * sp, oz = ct;
        float Y[9];
        sh9<float>(ox, oy, oz, Y);
        float Lc[3];
        for (int c = 0; c < 3; ++c) {
            float acc = 0.0f;
            for (int k = 0; k < 9; ++k) acc = fmaf(shs[9 * c + k], Y[k], acc);
            Lc[c] = acc;
        }
        tab[2 * (j - j0)] = make_float4(ox, oy, oz, st);
        tab[2 * (j - j0) + 1] = make_float4(st * Lc[0], st * Lc[1], st * Lc[2], 0.0f);
    }
}

// Unit normal of a Gaussian at (mx, my, mz) with rotation (qw, qx, qy, qz)
// and scales (s0, s1, s2): its smallest-scale axis (first on ties), turned
// away from the reference point c.
__device__ __forceinline__ float3 relight_axis_normal_v(float mx, float my, float mz, float qw, float qx,
                                                        float qy, float qz, float s0, float s1, float s2,
                                                        float cx, float cy, float cz) {
    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    int k = 0;
    float sm = s0;
    if (s1 < sm) { k = 1; sm = s1; }
    if (s2 < sm) k = 2;
    float nx, ny, nz;
    // column k of R(q): the Gaussian's k-th local axis
    if (k == 0) {
        nx = 1.f - 2.f * (qy * qy + qz * qz); ny = 2.f * (qx * qy + qw * qz); nz = 2.f * (qx * qz - qw * qy);
    } else if (k == 1) {
        nx = 2.f * (qx * qy - qw * qz); ny = 1.f - 2.f * (qx * qx + qz * qz); nz = 2.f * (qy * qz + qw * qx);
    } else {
        nx = 2.f * (qx * qz + qw * qy); ny = 2.f * (qy * qz - qw * qx); nz = 1.f - 2.f * (qx * qx + qy * qy);
    }
    const float side = nx * (mx - cx) + ny * (my - cy) + nz * (mz - cz);
    if (side < 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
    return make_float3(nx, ny, nz);
}

// The same for Gaussian g of the arrays.
__device__ __forceinline__ float3 relight_axis_normal(const float *__restrict__ means,
                                                      const float *__restrict__ quats,
                                                      const float *__restrict__ scales, int64_t g, float cx,
                                                      float cy, float cz) {
    return relight_axis_normal_v(means[3 * g], means[3 * g + 1], means[3 * g + 2], quats[4 * g], quats[4 * g + 1],
                                 quats[4 * g + 2], quats[4 * g + 3], scales[3 * g], scales[3 * g + 1],
                                 scales[3 * g + 2], cx, cy, cz);
}

// Eq. 10's sums over `count` table directions for RG normals n[r] at once
// (each table entry is read from shared memory once for all RG of them),
// added to acc[r] = (sum w L_r S, sum w L_g S, sum w L_b S, sum w S),
// S = max(0, omega.n[r])^q, in table order j = 0, 1, ... for every r.  A
// table split into consecutive pieces gives the same sums when the pieces
// are added in order.
template <int RG>
__device__ __forceinline__ void relight_accumulate_add(const float4 *tab, int count, float q,
                                                       const float3 (&n)[RG], float4 (&acc)[RG]) {
    if (q == 1.0f) {
#pragma unroll 2
        for (int j = 0; j < count; ++j) {
            const float4 a = tab[2 * j], b = tab[2 * j + 1];
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const float S = fmaxf(fmaf(a.x, n[r].x, fmaf(a.y, n[r].y, a.z * n[r].z)), 0.0f);
                acc[r].w = fmaf(S, a.w, acc[r].w);
                acc[r].x = fmaf(S, b.x, acc[r].x);
                acc[r].y = fmaf(S, b.y, acc[r].y);
                acc[r].z = fmaf(S, b.z, acc[r].z);
            }
        }
    } else {
        for (int j = 0; j < count; ++j) {
            const float4 a = tab[2 * j], b = tab[2 * j + 1];
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const float c = fmaf(a.x, n[r].x, fmaf(a.y, n[r].y, a.z * n[r].z));
                const float S = c > 0.0f ? exp2f(q * log2f(c)) : 0.0f;
                acc[r].w = fmaf(S, a.w, acc[r].w);
                acc[r].x = fmaf(S, b.x, acc[r].x);
                acc[r].y = fmaf(S, b.y, acc[r].y);
                acc[r].z = fmaf(S, b.z, acc[r].z);
            }
        }
    }
}

// The same sums over a whole table, from zero.
template <int RG>
__device__ __forceinline__ void relight_accumulate(const float4 *tab, int count, float q, const float3 (&n)[RG],
                                                   float4 (&acc)[RG]) {
#pragma unroll
    for (int r = 0; r < RG; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    relight_accumulate_add<RG>(tab, count, q, n, acc);
}

// Eqs. 9-10: the clipped transfer scale and the relit colour of Gaussian g
// from its colour (c0, c1, c2) before relighting.
__device__ __forceinline__ void relight_write_rgb(const float4 &acc, float eps, float t_max, float gamma, float c0,
                                                  float c1, float c2, float *cout, int64_t g) {
    const float inv = 1.0f / (acc.w + eps);
    const float sc0 = fminf(fmaxf(acc.x * inv, 0.0f), t_max);
    const float sc1 = fminf(fmaxf(acc.y * inv, 0.0f), t_max);
    const float sc2 = fminf(fmaxf(acc.z * inv, 0.0f), t_max);
    cout[3 * g] = fmaxf(gamma * c0 * sc0, 0.0f);
    cout[3 * g + 1] = fmaxf(gamma * c1 * sc1, 0.0f);
    cout[3 * g + 2] = fmaxf(gamma * c2 * sc2, 0.0f);
}

// The same with the colour read from cin (cin may equal cout).
__device__ __forceinline__ void relight_write(const float4 &acc, float eps, float t_max, float gamma,
                                              const float *cin, float *cout, int64_t g) {
    relight_write_rgb(acc, eps, t_max, gamma, cin[3 * g], cin[3 * g + 1], cin[3 * g + 2], cout, g);
}

}  // namespace
}  // namespace dgsm
