// build.cu -- Deep Gaussian Shadow Map build on sm_103a (Sec. 3.2).
//
// Pipeline per call (all on the caller's stream):
//   rect_cones_kernel   direction cones of every atlas tile and super-tile
//   prep_kernel         per (light, Gaussian): whitening matrix M = S^-1 R^T,
//                       w' = M (mu - o), beta (Eq. 5), culling radius, shell
//                       window and the binning cone
//   bin_count_kernel    tiles overlapped by each Gaussian's cone
//   scan                exclusive prefix sum -> pair offsets   (one host sync)
//   bin_emit_kernel     (key = light*tiles + tile, value = Gaussian) pairs
//   radix sort          stable, by key
//   tile_ranges_kernel  [start, end) of every key
//   build_tiles_kernel  per tile: stage the tile's Gaussians in shared
//                       memory, evaluate Eq. 3 per (texel ray, Gaussian,
//                       shell), prefix-sum over shells, T = exp(-tau) (Eq. 4)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int SUPER = 8;  // super-tile edge, in tiles

// Per (light, Gaussian) record read by the build kernel (64 bytes):
//   a = (M00 M01 M02 M10), b = (M11 M12 M20 M21), c = (M22 w'x w'y w'z),
//   d = (beta sqrt(pi/2), k^2, packed window, unused)
// packed window: bits 0-9 first shell of the window, 10-19 first shell past
// it, bit 20 = light inside the Gaussian's culling sphere.
struct __align__(16) BuildRec {
    float4 a, b, c, d;
};

// Per (light, Gaussian) binning record (32 bytes): a = (dir xyz, cos theta),
// b = (sin theta, mode, -, -); mode 0 = not binned, 1 = cone test, 2 = all tiles.
struct __align__(16) BinRec {
    float4 a, b;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void record_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Direction cone of the texel-centre rectangle [j0,j1) x [i0,i1): axis = the
// decoded centre of the rectangle, half-angle = the largest angle to the
// rectangle's corners, the points where its edges cross the fold lines
// u = 0, v = 0, |u| + |v| = 1, and (0,0) when inside.  Within each octant the
// decode is a central projection, so these vertices bound the angle.
// out: (axis xyz, cos), (sin, whole, -, -); whole = 1 when cos <= 0.
// ---------------------------------------------------------------------------
__device__ void rect_cone(int i0, int i1, int j0, int j1, int H, int W, float4 *out) {
    const float ua = xcentre(j0, W), ub = xcentre(j1 - 1, W);
    const float va = xcentre(i0, H), vb = xcentre(i1 - 1, H);
    const float uc = xmul(xadd(ua, ub), 0.5f), vc = xmul(xadd(va, vb), 0.5f);
    const float3 c = xdecode(uc, vc);
    float cmin = 1.0f;
    auto consider = [&](float u, float v) {
        float3 d = xdecode(u, v);
        float cs = xdot(c.x, c.y, c.z, d.x, d.y, d.z);
        cmin = fminf(cmin, cs);
    };
    consider(ua, va);
    consider(ub, va);
    consider(ua, vb);
    consider(ub, vb);
    for (int e = 0; e < 2; ++e) {
        const float y = e ? vb : va;
        const float cand[5] = {0.0f, xsub(1.0f, y), xsub(-1.0f, y), xadd(1.0f, y), xsub(y, 1.0f)};
#pragma unroll
        for (int m = 0; m < 5; ++m)
            if (ua <= cand[m] && cand[m] <= ub) consider(cand[m], y);
    }
    for (int e = 0; e < 2; ++e) {
        const float x = e ? ub : ua;
        const float cand[5] = {0.0f, xsub(1.0f, x), xsub(-1.0f, x), xadd(1.0f, x), xsub(x, 1.0f)};
#pragma unroll
        for (int m = 0; m < 5; ++m)
            if (va <= cand[m] && cand[m] <= vb) consider(x, cand[m]);
    }
    if (ua <= 0.0f && 0.0f <= ub && va <= 0.0f && 0.0f <= vb) consider(0.0f, 0.0f);
    if (cmin <= 0.0f) {
        out[0] = make_float4(c.x, c.y, c.z, -1.0f);
        out[1] = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
    } else {
        out[0] = make_float4(c.x, c.y, c.z, cmin);
        out[1] = make_float4(xsqrt(xsub(1.0f, xmul(cmin, cmin))), 0.0f, 0.0f, 0.0f);
    }
}

// cones: [0, n_tiles) tiles, then [n_tiles, n_tiles + n_super) super-tiles;
// two float4 per cone.
__global__ void rect_cones_kernel(int H, int W, int tile, int tx, int ty, int sx, int sy,
                                  float4 *__restrict__ cones) {
    const int n_tiles = tx * ty, n_super = sx * sy;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_tiles + n_super) return;
    int edge, a, b;
    if (idx < n_tiles) {
        edge = tile;
        a = idx / tx;
        b = idx % tx;
    } else {
        edge = tile * SUPER;
        a = (idx - n_tiles) / sx;
        b = (idx - n_tiles) % sx;
    }
    const int i0 = a * edge, j0 = b * edge;
    rect_cone(i0, min(i0 + edge, H), j0, min(j0 + edge, W), H, W, cones + 2 * idx);
}

// ---------------------------------------------------------------------------
// Per (light, Gaussian) preparation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prep_kernel(
    const float *__restrict__ means, const float *__restrict__ scales,
    const float *__restrict__ quats, const float *__restrict__ opac, int64_t N,
    const float *__restrict__ lights, int L, const float *__restrict__ radii, int K, float kappa,
    float eps, BuildRec *__restrict__ brec, BinRec *__restrict__ bin, int *__restrict__ status) {
    const int64_t total = (int64_t)L * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx / N);
        const int64_t g = idx - (int64_t)l * N;
        const float mx = means[3 * g], my = means[3 * g + 1], mz = means[3 * g + 2];
        const float s0 = scales[3 * g], s1 = scales[3 * g + 1], s2 = scales[3 * g + 2];
        // quats == nullptr: binning only (no build record)
        float qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f;
        if (quats) {
            qw = quats[4 * g]; qx = quats[4 * g + 1]; qy = quats[4 * g + 2]; qz = quats[4 * g + 3];
        }
        const float alpha = opac[g];
        const float ox = lights[3 * l], oy = lights[3 * l + 1], oz = lights[3 * l + 2];

        BinRec br;
        br.a = make_float4(0.f, 0.f, 1.f, -1.f);
        br.b = make_float4(0.f, 0.f, 0.f, 0.f);  // mode 0: not binned
        const bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(s0) &&
                            isfinite(s1) && isfinite(s2) && isfinite(qw) && isfinite(qx) &&
                            isfinite(qy) && isfinite(qz) && isfinite(alpha) && s0 > 0.f &&
                            s1 > 0.f && s2 > 0.f;
        if (!finite) {
            record_status(status, DGSM_ERR_NONFINITE_INPUT);
            bin[idx] = br;
            continue;
        }
        // --- binning specification (IEEE single ops, bit-exact with the CPU) ---
        float a = alpha;
        if (!(a > 0.0f)) {
            bin[idx] = br;
            continue;
        }
        a = fminf(a, 0.999999f);
        const float smax = fmaxf(fmaxf(s0, s1), s2);
        const float smin = fminf(fminf(s0, s1), s2);
        const float odds = xdiv(a, xsub(1.0f, a));
        const float Q = xdiv(xmul(xmul(kappa, odds), xdiv(smax, smin)), eps);
        int e = 0;
        frexpf(Q, &e);
        e = max(e, 1);
        const float k2 = xmul(1.38629436f, (float)e);
        const float r = xmul(xsqrt(k2), smax);
        const float vx = xsub(mx, ox), vy = xsub(my, oy), vz = xsub(mz, oz);
        const float dist = xsqrt(xadd(xadd(xmul(vx, vx), xmul(vy, vy)), xmul(vz, vz)));
        const float lo = xsub(dist, r);
        if (lo > radii[K - 1]) {
            bin[idx] = br;
            continue;
        }
        const bool inside = r >= dist;
        if (inside) {
            br.a = make_float4(0.f, 0.f, 1.f, -1.f);
            br.b = make_float4(0.f, 2.f, 0.f, 0.f);
        } else {
            const float sn = xdiv(r, dist);
            const float cs = xsqrt(xsub(1.0f, xmul(sn, sn)));
            br.a = make_float4(xdiv(vx, dist), xdiv(vy, dist), xdiv(vz, dist), cs);
            br.b = make_float4(sn, 1.f, 0.f, 0.f);
        }
        bin[idx] = br;
        if (!quats) continue;

        // --- build record (ordinary single precision) ---
        const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw *= qn; qx *= qn; qy *= qn; qz *= qn;
        // rotation matrix columns are the Gaussian's local axes
        const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz),
                    R02 = 2.f * (qx * qz + qw * qy);
        const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz),
                    R12 = 2.f * (qy * qz - qw * qx);
        const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx),
                    R22 = 1.f - 2.f * (qx * qx + qy * qy);
        const float i0 = 1.f / s0, i1 = 1.f / s1, i2 = 1.f / s2;
        // M = S^-1 R^T: row k = (column k of R) / s_k, so A = M^T M
        const float M00 = R00 * i0, M01 = R10 * i0, M02 = R20 * i0;
        const float M10 = R01 * i1, M11 = R11 * i1, M12 = R21 * i1;
        const float M20 = R02 * i2, M21 = R12 * i2, M22 = R22 * i2;
        const float wx = M00 * vx + M01 * vy + M02 * vz;
        const float wy = M10 * vx + M11 * vy + M12 * vz;
        const float wz = M20 * vx + M21 * vy + M22 * vz;
        const float tau_star = -log1pf(-a);
        const float trA = i0 * i0 + i1 * i1 + i2 * i2;
        // beta sqrt(pi/2) = kappa tau* sqrt(tr A / 3) / sqrt(2 pi) * sqrt(pi/2)
        const float bpref = 0.5f * kappa * tau_star * sqrtf(trA * (1.0f / 3.0f));
        const float hi = dist + r;
        int klo = 0, kend = 0;
        if (!inside) {
            while (klo < K && radii[klo] < lo) ++klo;
        }
        kend = klo;
        while (kend < K && radii[kend] <= hi) ++kend;
        const int packed = klo | (kend << 10) | ((inside ? 1 : 0) << 20);
        BuildRec rec;
        rec.a = make_float4(M00, M01, M02, M10);
        rec.b = make_float4(M11, M12, M20, M21);
        rec.c = make_float4(M22, wx, wy, wz);
        rec.d = make_float4(bpref, k2, __int_as_float(packed), 0.f);
        brec[idx] = rec;
    }
}

__device__ __forceinline__ bool cone_overlap(const BinRec &g, const float4 *cone) {
    const float4 c0 = __ldg(cone), c1 = __ldg(cone + 1);
    if (c1.y != 0.0f) return true;  // cone spans a hemisphere
    const float dot = xdot(g.a.x, g.a.y, g.a.z, c0.x, c0.y, c0.z);
    const float rhs = xsub(xmul(g.a.w, c0.w), xmul(g.b.x, c1.x));
    return dot >= rhs;
}

// Count (emit = false) or write (emit = true) the tiles each Gaussian overlaps.
template <bool EMIT>
__global__ void __launch_bounds__(256) bin_tiles_kernel(
    const BinRec *__restrict__ bin, int64_t N, int L, int tx, int ty, int sx, int sy,
    const float4 *__restrict__ cones, uint32_t *__restrict__ counts,
    const uint32_t *__restrict__ offsets, uint32_t *__restrict__ keys,
    uint32_t *__restrict__ vals) {
    const int64_t total = (int64_t)L * N;
    const int n_tiles = tx * ty;
    const float4 *scones = cones + 2 * n_tiles;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const BinRec g = bin[idx];
        const int mode = (int)g.b.y;
        const int l = (int)(idx / N);
        const uint32_t gi = (uint32_t)(idx - (int64_t)l * N);
        uint32_t c = 0, off = 0;
        if (EMIT) off = offsets[idx];
        if (mode == 2) {
            if (EMIT) {
                for (int t = 0; t < n_tiles; ++t) {
                    keys[off + t] = (uint32_t)(l * n_tiles + t);
                    vals[off + t] = gi;
                }
            }
            c = n_tiles;
        } else if (mode == 1) {
            for (int sa = 0; sa < sy; ++sa)
                for (int sb = 0; sb < sx; ++sb) {
                    if (!cone_overlap(g, scones + 2 * (sa * sx + sb))) continue;
                    const int a1 = min(sa * SUPER + SUPER, ty), b1 = min(sb * SUPER + SUPER, tx);
                    for (int a = sa * SUPER; a < a1; ++a)
                        for (int b = sb * SUPER; b < b1; ++b) {
                            const int t = a * tx + b;
                            if (!cone_overlap(g, cones + 2 * t)) continue;
                            if (EMIT) {
                                keys[off + c] = (uint32_t)(l * n_tiles + t);
                                vals[off + c] = gi;
                            }
                            ++c;
                        }
                }
        }
        if (!EMIT) counts[idx] = c;
    }
}

__global__ void tile_ranges_kernel(const uint32_t *__restrict__ keys, int64_t P,
                                   uint32_t *__restrict__ start, uint32_t *__restrict__ end) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[p];
        if (p == 0 || keys[p - 1] != k) start[k] = (uint32_t)p;
        if (p == P - 1 || keys[p + 1] != k) end[k] = (uint32_t)(p + 1);
    }
}

template <typename T>
__device__ __forceinline__ T to_store(float x);
template <>
__device__ __forceinline__ float to_store<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half to_store<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}

// erfc(y) for y >= 0 by Abramowitz & Stegun 7.1.26 (after Hastings):
// erfc(y) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-y^2), t = 1/(1 + p y),
// |error| <= 1.5e-7.  mass_below(x) returns A0 em erfc(-x) =
// int_-inf^t of the Gaussian along the ray, with x = sqrt(a/2)(t - s*),
// `full` = 2 A0 em the integral over the whole line and hm2 = -m^2/2 log2(e).
__device__ __forceinline__ float mass_below(float x, float A0, float hm2, float full) {
    constexpr float P = 0.3275911f;
    constexpr float A1 = 0.254829592f, A2 = -0.284496736f, A3 = 1.421413741f,
                    A4 = -1.453152027f, A5 = 1.061405429f;
    constexpr float LOG2E = 1.4426950408889634f;
    const float y = fabsf(x);
    const float t = rcp_approx(fmaf(P, y, 1.0f));
    const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, A5, A4), A3), A2), A1);
    const float e = ex2_approx(fmaf(-y * LOG2E, y, hm2));
    const float tail = A0 * poly * e;
    return x >= 0.0f ? full - tail : tail;
}

// One block per (light, tile); one thread per texel of the tile.
template <typename OutT>
__global__ void __launch_bounds__(256) build_tiles_kernel(
    const BuildRec *__restrict__ brec, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ tstart, const uint32_t *__restrict__ tend,
    const float *__restrict__ radii, int K, int H, int W, int tile, int tx, int n_tiles,
    int64_t N, int chunk, OutT *__restrict__ atlas, unsigned long long *__restrict__ stats) {
    extern __shared__ float4 smem4[];
    const int nt = tile * tile;
    float4 *stage = smem4;                              // chunk x 4 float4
    float *D = reinterpret_cast<float *>(smem4 + 4 * chunk);  // K x nt shell increments
    float *rs = D + K * nt;                             // K radii
    const int key = blockIdx.x;
    const int l = key / n_tiles, t = key - l * n_tiles;
    const int tile_i = t / tx, tile_j = t - tile_i * tx;
    const int tid = threadIdx.x;
    const int i = tile_i * tile + tid / tile, j = tile_j * tile + tid % tile;
    const bool valid = i < H && j < W;
    for (int k = 0; k < K; ++k) D[k * nt + tid] = 0.0f;
    for (int k = tid; k < K; k += nt) rs[k] = radii[k];
    // texel ray direction: decoded texel centre
    const float u = (2.0f * j + 1.0f) / W - 1.0f, v = (2.0f * i + 1.0f) / H - 1.0f;
    float z = 1.0f - fabsf(u) - fabsf(v), x = u, y = v;
    if (z < 0.0f) {
        x = copysignf(1.0f - fabsf(v), u >= 0.f ? 1.f : -1.f);
        y = copysignf(1.0f - fabsf(u), v >= 0.f ? 1.f : -1.f);
    }
    const float inv = rsqrtf(x * x + y * y + z * z);
    const float dx = x * inv, dy = y * inv, dz = z * inv;

    const uint32_t p0 = tstart[key], p1 = tend[key];
    unsigned long long n_hit = 0, n_shell = 0;
    __syncthreads();
    for (uint32_t base = p0; base < p1; base += chunk) {
        const int cnt = (int)min((uint32_t)chunk, p1 - base);
        const float4 *src = reinterpret_cast<const float4 *>(brec) + (int64_t)l * N * 4;
        for (int e = tid; e < cnt * 4; e += nt) {
            const uint32_t g = vals[base + (e >> 2)];
            stage[e] = __ldg(src + (int64_t)g * 4 + (e & 3));
        }
        __syncthreads();
        if (valid) {
            for (int r = 0; r < cnt; ++r) {
                const float4 q0 = stage[4 * r], q1 = stage[4 * r + 1], q2 = stage[4 * r + 2],
                             q3 = stage[4 * r + 3];
                // whitened ray direction d' = M d
                const float px = fmaf(q0.x, dx, fmaf(q0.y, dy, q0.z * dz));
                const float py = fmaf(q0.w, dx, fmaf(q1.x, dy, q1.y * dz));
                const float pz = fmaf(q1.z, dx, fmaf(q1.w, dy, q2.x * dz));
                const float wx = q2.y, wy = q2.z, wz = q2.w;
                const float a = fmaf(px, px, fmaf(py, py, pz * pz));      // d^T A d
                const float pw = fmaf(px, wx, fmaf(py, wy, pz * wz));     // -b
                const float cx = fmaf(wy, pz, -wz * py);                  // w' x d'
                const float cy = fmaf(wz, px, -wx * pz);
                const float cz = fmaf(wx, py, -wy * px);
                const float c2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                const float ia = rcp_approx(a);
                const float m2 = c2 * ia;   // c - b^2/a without cancellation
                const float ss = pw * ia;   // closest approach s* = -b/a
                const int packed = __float_as_int(q3.z);
                const bool inside = (packed >> 20) & 1;
                if (m2 <= q3.y && (inside || ss > 0.0f)) {
                    const int klo = packed & 1023, kend = (packed >> 10) & 1023;
                    ++n_hit;
                    n_shell += kend - klo;
                    const float rsa = rsqrt_approx(a);
                    const float A0 = q3.x * rsa;                 // beta sqrt(pi/(2a))
                    const float h = a * rsa * 0.70710678118f;    // sqrt(a/2)
                    const float hm2 = -0.72134752044f * m2;      // -m^2/2 log2(e)
                    const float full = 2.0f * A0 * ex2_approx(hm2);
                    const float hs = h * ss;
                    const float F0 = inside ? mass_below(-hs, A0, hm2, full) : 0.0f;
                    float Gprev = 0.0f;
                    for (int k = klo; k < kend; ++k) {
                        const float G = mass_below(fmaf(h, rs[k], -hs), A0, hm2, full) - F0;
                        D[k * nt + tid] += fmaxf(G - Gprev, 0.0f);
                        Gprev = fmaxf(G, Gprev);
                    }
                    if (kend < K) D[kend * nt + tid] += fmaxf(full - F0 - Gprev, 0.0f);
                }
            }
        }
        __syncthreads();
    }
    if (valid) {
        float tau = 0.0f, Tprev = 1.0f;
        const int64_t plane = (int64_t)H * W;
        OutT *dst = atlas + (int64_t)l * K * plane + (int64_t)i * W + j;
        for (int k = 0; k < K; ++k) {
            tau += D[k * nt + tid];
            const float T = fminf(expf(-tau), Tprev);  // Eq. 4, kept non-increasing in k
            Tprev = T;
            dst[k * plane] = to_store<OutT>(T);
        }
    }
    if (stats) {
        // block counters in shared memory (blocks of 16 threads fill half a warp)
        __shared__ unsigned long long cnt[2];
        if (tid == 0) cnt[0] = cnt[1] = 0ull;
        __syncthreads();
        if (n_hit) atomicAdd(&cnt[0], n_hit);
        if (n_shell) atomicAdd(&cnt[1], n_shell);
        __syncthreads();
        if (tid == 0) {
            const int nvalid = (min(tile_i * tile + tile, H) - tile_i * tile) *
                               (min(tile_j * tile + tile, W) - tile_j * tile);
            atomicAdd(stats + 0, (unsigned long long)nvalid * (p1 - p0));
            atomicAdd(stats + 1, cnt[0]);
            atomicAdd(stats + 2, cnt[1]);
        }
    }
}

size_t build_smem_bytes(int K, int tile, int chunk) {
    return (size_t)chunk * 4 * sizeof(float4) + (size_t)K * tile * tile * sizeof(float) +
           (size_t)K * sizeof(float);
}

template <typename OutT>
int launch_build_tiles(dgsm_ctx *ctx, const BuildRec *brec, const uint32_t *vals,
                       const uint32_t *ts, const uint32_t *te, const float *radii, int K, int H,
                       int W, int tile, int tx, int n_tiles, int L, int64_t N, int chunk, void *atlas,
                       cudaStream_t s) {
    size_t smem = build_smem_bytes(K, tile, chunk);
    cudaError_t e = cudaFuncSetAttribute(build_tiles_kernel<OutT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: smem attribute");
    build_tiles_kernel<OutT><<<L * n_tiles, tile * tile, smem, s>>>(
        brec, vals, ts, te, radii, K, H, W, tile, tx, n_tiles, N, chunk, (OutT *)atlas,
        ctx->d_stats);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "build_tiles_kernel");
}

struct BinOut {
    int64_t P = 0;
    uint32_t *keys = nullptr, *vals = nullptr;
    uint32_t *ts = nullptr, *te = nullptr;
    BuildRec *brec = nullptr;
    int tx = 0, ty = 0, n_tiles = 0;
};

int check_common(dgsm_ctx *ctx, const float *means, const float *scales, const float *opac,
                 int64_t n, const float *lights, int L, int H, int W, const float *radii, int K,
                 const dgsm_params &p) {
    if (n < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!means || !scales || !opac))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "null Gaussian array");
    if (n >= (int64_t)1 << 31) return fail(ctx, DGSM_ERR_INVALID_ARG, "n >= 2^31");
    if (!lights || L < 1 || L > 64) return fail(ctx, DGSM_ERR_INVALID_ARG, "need 1..64 lights");
    if (H < 1 || W < 1 || H > 4096 || W > 4096) return fail(ctx, DGSM_ERR_INVALID_ARG, "H, W must be in 1..4096");
    if (!radii || K < 1 || K > 256) return fail(ctx, DGSM_ERR_INVALID_ARG, "K must be in 1..256");
    if (p.tile != 4 && p.tile != 8 && p.tile != 16) return fail(ctx, DGSM_ERR_INVALID_ARG, "tile must be 4, 8 or 16");
    if (p.chunk < 16 || p.chunk > 256) return fail(ctx, DGSM_ERR_INVALID_ARG, "chunk must be in 16..256");
    if (!(p.kappa >= 0.f) || !(p.eps_cull > 0.f)) return fail(ctx, DGSM_ERR_INVALID_ARG, "kappa >= 0 and eps_cull > 0 required");
    if (build_smem_bytes(K, p.tile, p.chunk) > 220 * 1024)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "K x tile^2 too large for shared memory: use a smaller tile");
    return DGSM_OK;
}

// prep + binning + sort + ranges.  Blocks once to read the pair count.
int run_binning(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                const float *opac, int64_t N, const float *lights, int L, int H, int W,
                const float *radii, int K, const dgsm_params &p, cudaStream_t s, BinOut *out) {
    const int tile = p.tile;
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    const int sx = (tx + SUPER - 1) / SUPER, sy = (ty + SUPER - 1) / SUPER;
    const int n_tiles = tx * ty;
    out->tx = tx; out->ty = ty; out->n_tiles = n_tiles;
    const int64_t LN = (int64_t)L * N;
    const int64_t nkeys = (int64_t)L * n_tiles;
    void *w_br, *w_bin, *w_cnt, *w_cones, *w_rng;
    int rc;
    if ((rc = ws_reserve(ctx, WS_BUILD_REC, sizeof(BuildRec) * (size_t)LN, &w_br))) return rc;
    if ((rc = ws_reserve(ctx, WS_BIN_REC, sizeof(BinRec) * (size_t)LN, &w_bin))) return rc;
    if ((rc = ws_reserve(ctx, WS_COUNTS, sizeof(uint32_t) * (size_t)LN, &w_cnt))) return rc;
    if ((rc = ws_reserve(ctx, WS_CONES, 2 * sizeof(float4) * (size_t)(n_tiles + sx * sy), &w_cones))) return rc;
    if ((rc = ws_reserve(ctx, WS_RANGES, 2 * sizeof(uint32_t) * (size_t)nkeys, &w_rng))) return rc;
    out->brec = (BuildRec *)w_br;
    out->ts = (uint32_t *)w_rng;
    out->te = out->ts + nkeys;
    cudaError_t e = cudaMemsetAsync(w_rng, 0, 2 * sizeof(uint32_t) * (size_t)nkeys, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_stats, 0, 8 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: memset");
    out->P = 0;
    if (N == 0) return DGSM_OK;

    const int nc = n_tiles + sx * sy;
    rect_cones_kernel<<<(nc + 127) / 128, 128, 0, s>>>(H, W, tile, tx, ty, sx, sy, (float4 *)w_cones);
    const int grid = (int)std::min<int64_t>((LN + 255) / 256, (int64_t)ctx->num_sms * 16);
    prep_kernel<<<grid, 256, 0, s>>>(means, scales, quats, opac, N, lights, L, radii, K, p.kappa,
                                     p.eps_cull, (BuildRec *)w_br, (BinRec *)w_bin, ctx->d_status);
    bin_tiles_kernel<false><<<grid, 256, 0, s>>>((const BinRec *)w_bin, N, L, tx, ty, sx, sy,
                                                  (const float4 *)w_cones, (uint32_t *)w_cnt,
                                                  nullptr, nullptr, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "prep/count kernels");
    if ((rc = scan_exclusive_u32(ctx, (uint32_t *)w_cnt, (uint32_t *)w_cnt, LN, ctx->d_stats + 3, s)))
        return rc;
    e = cudaMemcpyAsync(ctx->h_pinned, ctx->d_stats + 3, sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned + 1, ctx->d_status, sizeof(int),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build: pair count");
    const int st = *(int *)(ctx->h_pinned + 1);
    if (st != DGSM_OK) {
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
        return fail(ctx, st, "a Gaussian has a non-finite field or a non-positive scale");
    }
    const unsigned long long P = ctx->h_pinned[0];
    if (P >= (1ull << 31)) return fail(ctx, DGSM_ERR_WORKSPACE, "more than 2^31 binned pairs");
    out->P = (int64_t)P;
    if (P == 0) return DGSM_OK;
    void *ka, *va, *kb, *vb;
    if ((rc = ws_reserve(ctx, WS_KEYS_A, sizeof(uint32_t) * P, &ka))) return rc;
    if ((rc = ws_reserve(ctx, WS_VALS_A, sizeof(uint32_t) * P, &va))) return rc;
    if ((rc = ws_reserve(ctx, WS_KEYS_B, sizeof(uint32_t) * P, &kb))) return rc;
    if ((rc = ws_reserve(ctx, WS_VALS_B, sizeof(uint32_t) * P, &vb))) return rc;
    bin_tiles_kernel<true><<<grid, 256, 0, s>>>((const BinRec *)w_bin, N, L, tx, ty, sx, sy,
                                                 (const float4 *)w_cones, nullptr,
                                                 (const uint32_t *)w_cnt, (uint32_t *)ka,
                                                 (uint32_t *)va);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bin emit kernel");
    int bits = 0;
    while (bits < 32 && ((uint64_t)(nkeys - 1) >> bits) != 0) ++bits;
    uint32_t *keys = (uint32_t *)ka, *vals = (uint32_t *)va;
    if ((rc = radix_sort_pairs(ctx, &keys, &vals, (uint32_t *)kb, (uint32_t *)vb, (int64_t)P, bits, s)))
        return rc;
    const int rgrid = (int)std::min<int64_t>(((int64_t)P + 255) / 256, (int64_t)ctx->num_sms * 16);
    tile_ranges_kernel<<<rgrid, 256, 0, s>>>(keys, (int64_t)P, out->ts, out->te);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile ranges kernel");
    out->keys = keys;
    out->vals = vals;
    return DGSM_OK;
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_build(dgsm_ctx *ctx, const float *means, const float *scales,
                          const float *quats, const float *opac, int64_t n, const float *lights,
                          int32_t L, int32_t H, int32_t W, const float *radii, int32_t K,
                          const dgsm_params *params, void *atlas, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    int rc = check_common(ctx, means, scales, opac, n, lights, L, H, W, radii, K, p);
    if (rc) return rc;
    if (n > 0 && !quats) return fail(ctx, DGSM_ERR_INVALID_ARG, "null quats");
    if (!atlas) return fail(ctx, DGSM_ERR_INVALID_ARG, "null atlas");
    if (p.atlas_dtype < DGSM_F32 || p.atlas_dtype > DGSM_BF16)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "atlas_dtype must be DGSM_F32, DGSM_F16 or DGSM_BF16");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    BinOut b;
    if ((rc = run_binning(ctx, means, scales, quats, opac, n, lights, L, H, W, radii, K, p, s, &b)))
        return rc;
    const uint32_t *vals = b.vals ? b.vals : b.ts;  // unused when there are no pairs
    switch (p.atlas_dtype) {
        case DGSM_F32:
            rc = launch_build_tiles<float>(ctx, b.brec, vals, b.ts, b.te, radii, K, H, W, p.tile,
                                           b.tx, b.n_tiles, L, n, p.chunk, atlas, s);
            break;
        case DGSM_F16:
            rc = launch_build_tiles<__half>(ctx, b.brec, vals, b.ts, b.te, radii, K, H, W, p.tile,
                                            b.tx, b.n_tiles, L, n, p.chunk, atlas, s);
            break;
        default:
            rc = launch_build_tiles<__nv_bfloat16>(ctx, b.brec, vals, b.ts, b.te, radii, K, H, W,
                                                   p.tile, b.tx, b.n_tiles, L, n, p.chunk, atlas, s);
    }
    if (rc) return rc;
    ctx->h_pinned[8] = (unsigned long long)b.P;  // pair count of this build
    return DGSM_OK;
}

extern "C" int dgsm_get_build_stats(dgsm_ctx *ctx, dgsm_build_stats *out) {
    if (!ctx || !out) return DGSM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(ctx->h_pinned + 4, ctx->d_stats, 3 * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dgsm_get_build_stats");
    out->n_pairs = (int64_t)ctx->h_pinned[8];
    out->rays_tested = (int64_t)ctx->h_pinned[4];
    out->ray_evals = (int64_t)ctx->h_pinned[5];
    out->shell_evals = (int64_t)ctx->h_pinned[6];
    return DGSM_OK;
}

extern "C" int dgsm_bin(dgsm_ctx *ctx, const float *means, const float *scales, const float *opac,
                        int64_t n, const float *lights, int32_t L, int32_t H, int32_t W,
                        const float *radii, int32_t K, const dgsm_params *params,
                        uint32_t *keys_out, uint32_t *vals_out, int64_t capacity,
                        int64_t *n_pairs_out, void *stream) {
    if (!ctx || !n_pairs_out) return DGSM_ERR_INVALID_ARG;
    dgsm_params p;
    if (params) p = *params; else dgsm_default_params(&p);
    int rc = check_common(ctx, means, scales, opac, n, lights, L, H, W, radii, K, p);
    if (rc) return rc;
    if (capacity < 0 || (capacity > 0 && (!keys_out || !vals_out)))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "bad output capacity or pointers");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    // binning never reads the quaternions (quats = nullptr skips the build records)
    BinOut b;
    if ((rc = run_binning(ctx, means, scales, nullptr, opac, n, lights, L, H, W, radii, K, p, s, &b)))
        return rc;
    *n_pairs_out = b.P;
    if (b.P > capacity) return fail(ctx, DGSM_ERR_WORKSPACE, "capacity smaller than the pair count");
    if (b.P > 0) {
        e = cudaMemcpyAsync(keys_out, b.keys, sizeof(uint32_t) * b.P, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals_out, b.vals, sizeof(uint32_t) * b.P, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dgsm_bin copy-out");
    return DGSM_OK;
}
