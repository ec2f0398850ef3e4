// attenuate.cu -- receiver attenuation by centre lookup (Sec. 3.3) on sm_103a.
//
// Per query Gaussian and light: octahedral code of (x - o_l)
// (exact single-precision index decisions, shared with dgsm_sample_index),
// bilinear between texel centres with clamp-to-edge, linear between the two
// shells bracketing t; the direct part of the colour is scaled by the
// light-weighted transmittance.  The pass streams 36 bytes per query
// (mean, colour in, colour out) and gathers 8 atlas taps per light.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "dgsm_internal.cuh"
#include "lookup.cuh"

namespace dgsm {
namespace {

constexpr int ATT_THREADS = 256;
constexpr int ATT_U = 4;  // queries in flight per thread

// Each block takes ATT_U * 256 consecutive queries; thread t handles queries
// t, t + 256, ... of the block's range, so every load and store instruction
// of a warp touches one contiguous span.  The ATT_U independent queries per
// thread keep several gathers and stream loads in flight (the pass is bound
// by memory latency unless enough requests are outstanding).
// SEP: the dynamic atlas has its own resolution and shells (Hd, Wd, Kd,
// radii_d) and is sampled at its own index; otherwise it shares the static
// atlas's geometry and index.
struct DynGeom {
    int H, W, K;
    const float *radii;
};

template <typename T, bool SEP, bool CUBE = false>
__global__ void __launch_bounds__(ATT_THREADS) attenuate_kernel(
    const T *__restrict__ atlas, const T *__restrict__ dyn, int L, int H, int W,
    const float *__restrict__ radii, int K, DynGeom dg, const float *__restrict__ lights,
    const float *__restrict__ qm, const float *cin, int64_t Q, const float *__restrict__ lw,
    float wd, float *cout, float *__restrict__ Tout) {
    __shared__ float rs[256], inw[256];
    __shared__ float rsd[SEP ? 256 : 1], inwd[SEP ? 256 : 1];
    __shared__ short tab[SHELL_BINS], tabd[SEP ? SHELL_BINS : 1];
    __shared__ float ls[64 * 3];
    __shared__ float wl[64];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        rs[k] = radii[k];
        inw[k] = k + 1 < K ? 1.0f / (radii[k + 1] - radii[k]) : 0.0f;
    }
    if (SEP)
        for (int k = threadIdx.x; k < dg.K; k += blockDim.x) {
            rsd[k] = dg.radii[k];
            inwd[k] = k + 1 < dg.K ? 1.0f / (dg.radii[k + 1] - dg.radii[k]) : 0.0f;
        }
    for (int k = threadIdx.x; k < 3 * L; k += blockDim.x) ls[k] = lights[k];
    for (int k = threadIdx.x; k < L; k += blockDim.x) wl[k] = lw ? lw[k] : 1.0f / (float)L;
    __syncthreads();
    const ShellTab st = build_shell_tab(rs, K, tab);
    ShellTab std_ = st;
    if (SEP) std_ = build_shell_tab(rsd, dg.K, tabd);
    __syncthreads();
    const int64_t lstride = (int64_t)K * H * W;
    const int64_t dstride = SEP ? (int64_t)dg.K * dg.H * dg.W : lstride;
    const int64_t span = (int64_t)ATT_U * ATT_THREADS;
    for (int64_t base = (int64_t)blockIdx.x * span; base < Q; base += (int64_t)gridDim.x * span) {
        float px[ATT_U], py[ATT_U], pz[ATT_U], c0[ATT_U], c1[ATT_U], c2[ATT_U], acc[ATT_U];
#pragma unroll
        for (int u = 0; u < ATT_U; ++u) {
            const int64_t q = base + u * ATT_THREADS + threadIdx.x;
            const bool ok = q < Q;
            px[u] = ok ? __ldg(qm + 3 * q) : 0.f;
            py[u] = ok ? __ldg(qm + 3 * q + 1) : 0.f;
            pz[u] = ok ? __ldg(qm + 3 * q + 2) : 0.f;
            c0[u] = ok ? cin[3 * q] : 0.f;
            c1[u] = ok ? cin[3 * q + 1] : 0.f;
            c2[u] = ok ? cin[3 * q + 2] : 0.f;
            acc[u] = 0.f;
        }
        for (int l = 0; l < L; ++l) {
            float Tl[ATT_U];
#pragma unroll
            for (int u = 0; u < ATT_U; ++u) {
                const float ox = ls[3 * l], oy = ls[3 * l + 1], oz = ls[3 * l + 2];
                const SampleIndex s = CUBE ? sample_index_cube(px[u], py[u], pz[u], ox, oy, oz, W, rs, K, tab, st)
                                           : sample_index_tab(px[u], py[u], pz[u], ox, oy, oz, H, W, rs, K, tab, st);
                Tl[u] = 1.0f;
                if (s.t != 0.0f) {
                    Tl[u] = lookup(atlas + l * lstride, H, W, K, s, rs, inw);
                    if (dyn) {
                        if (SEP) {
                            const SampleIndex sd = sample_index_tab(px[u], py[u], pz[u], ox, oy, oz, dg.H,
                                                                    dg.W, rsd, dg.K, tabd, std_);
                            Tl[u] *= lookup(dyn + l * dstride, dg.H, dg.W, dg.K, sd, rsd, inwd);
                        } else {
                            Tl[u] *= lookup(dyn + l * dstride, H, W, K, s, rs, inw);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < ATT_U; ++u) {
                const int64_t q = base + u * ATT_THREADS + threadIdx.x;
                if (Tout && q < Q) Tout[q * L + l] = Tl[u];
                acc[u] = fmaf(wl[l], Tl[u], acc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < ATT_U; ++u) {
            const int64_t q = base + u * ATT_THREADS + threadIdx.x;
            if (q >= Q) continue;
            const float f = 1.0f - wd + wd * acc[u];
            __stcs(cout + 3 * q, c0[u] * f);
            __stcs(cout + 3 * q + 1, c1[u] * f);
            __stcs(cout + 3 * q + 2, c2[u] * f);
        }
    }
}

// ---- streamed form for the octahedral atlas ---------------------------------
//
// The same lookup in another form, for the common case (octahedral map, at
// least 2 x 2 texels and 2 shells; no dynamic atlas, or one of the static
// atlas's geometry):
// * Streams by the bulk-copy engine.  A warp takes rounds of AZ_R
//   consecutive receivers.  One lane copies a round's means into the warp's
//   slice of shared memory with cp.async.bulk (completing on the warp's
//   mbarrier, a round ahead of its use, two stages), the lanes read them
//   there, write the attenuated colours over them (the input colours read
//   directly, once, at that point) and one bulk store sends them out.  The
//   slice stays small (3 KB per warp), leaving the L1 most of the SM's
//   on-chip memory for the atlas taps.  A round that is not whole (the last
//   one) or arrays that are not 16-byte aligned go through plain loads.
// * Shell index without a square root.  sqrt_rn is monotone, so
//   r_k <= sqrt_rn(d2) exactly when d2 >= thr_k, thr_k the smallest float
//   whose rounded square root reaches r_k.  A per-block table over the bits
//   of d2 (32 buckets per octave of d2 in [2^-24, 2^24) m^2) gives the count
//   in one step when no bucket holds two thresholds (else the thresholds are
//   counted one by one), so k equals the specification's
//   #{r_k <= sqrt_rn(d2)} - 1.  t itself enters only the shell weight, where
//   d2 rsqrt(d2) (within a few ulps of sqrt_rn(d2)) serves.
// * Edge taps by clamped weights.  Clamp-to-edge (j0 = j1 at a border) is
//   the same value as the pair (0, 1) with weight 0 or (W-2, W-1) with
//   weight 1, and likewise for rows and for the shells below the first or
//   past the last radius; so every lookup reads the taps (i0 + {0,1},
//   j0 + {0,1}, k0 + {0,1}) at fixed offsets from one address.
// * Both quotients of the octahedral code by one rounded reciprocal
//   y = RN(1/s) and Markstein's correction q = RN(q0 + RN(a - s q0) y),
//   q0 = RN(a y) (P. Markstein, IBM J. Res. Dev. 34(1), 1990): the correctly
//   rounded a / s of the specification away from underflow, and within an
//   ulp of it otherwise; the lookup is continuous across texel and shell
//   boundaries, so the result moves by at most that much where the texel
//   base would differ.
// * Two receivers per packed operation.  A lane's receivers u = 2p, 2p + 1
//   go through the floating-point steps as the two halves of f32x2
//   operations (fma/add/mul.rn.f32x2, each half rounded as the scalar
//   operation, x - o as fma(o, -1, x)), which halves the issue slots of the
//   arithmetic; the integer decisions, the reciprocal and the taps stay per
//   receiver.
// The texel base and the bilinear fractions are otherwise the
// specification's single-precision operations, as in sample_index_tab.
constexpr int AZ_THREADS = 512;     // two blocks per SM
constexpr int AZ_WARPS = AZ_THREADS / 32;
constexpr int AZ_U = 6;             // receivers per lane per round
constexpr int AZ_R = 32 * AZ_U;     // receivers per warp round
constexpr int AZ_BYTES = AZ_R * 12; // one round of one (n, 3) float array
constexpr int AZ_TB0 = 103 << 23;   // float bits of 2^-24 (d2 in m^2)
constexpr int AZ_NB = 1536;         // 32 buckets per octave of d2 over [2^-24, 2^24)
constexpr int AZ_SHIFT = 18;
constexpr long long AZ_WAIT = 2000000000ll;  // clock cycles before a wait gives up (about 1 s)
constexpr size_t AZ_SMEM = (size_t)AZ_WARPS * 2 * AZ_BYTES;  // per warp: two stages of means

__device__ __forceinline__ uint32_t az_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Phase `parity` of the mbarrier at `bar` completed; false after AZ_WAIT cycles.
__device__ __forceinline__ bool az_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > AZ_WAIT) return false;
    }
}

// One round's means into a stage (one lane), completing on bar.
__device__ __forceinline__ void az_issue(float *stg, const float *qm, int64_t base, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(AZ_BYTES) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(az_smem(stg)), "l"(qm + 3 * base), "r"(AZ_BYTES), "r"(bar) : "memory");
}

template <typename T, bool DYN, bool HAS_T>
__global__ void __launch_bounds__(AZ_THREADS, 2) attenuate_stream_kernel(
    const T *__restrict__ atlas, const T *__restrict__ dyn, int L, int H, int W,
    const float *__restrict__ radii, int K, const float *__restrict__ lights,
    const float *qm, const float *cin, int64_t Q, const float *__restrict__ lw, float wd,
    float *cout, float *__restrict__ Tout, bool vec, int *status) {
    // vec: qm, cin and cout are 16-byte aligned (whole rounds move by bulk copies)
    extern __shared__ __align__(16) float az_stage[];  // [warp][stage][3 AZ_R]: means, then colours out
    __shared__ float rs[256], inw[256], thr[257];
    __shared__ uint16_t dtab[AZ_NB];
    __shared__ float ls[64 * 3];
    __shared__ float wl[64];
    __shared__ __align__(8) unsigned long long bars[AZ_WARPS][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *slice = az_stage + (size_t)warp * 2 * 3 * AZ_R;
    const uint32_t bar0 = az_smem(&bars[warp][0]);
    const int64_t nwarps = (int64_t)gridDim.x * AZ_WARPS;
    auto whole = [&](int64_t b) { return vec && b + AZ_R <= Q; };
    int64_t base = ((int64_t)blockIdx.x * AZ_WARPS + warp) * AZ_R;
    // the warp's barriers, and its first round's copy in flight during the set-up
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (base < Q && whole(base)) az_issue(slice, qm, base, bar0);
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const float r = radii[k];
        rs[k] = r;
        inw[k] = k + 1 < K ? 1.0f / (radii[k + 1] - r) : 0.0f;
        // the smallest d with sqrt_rn(d) >= r
        float d = __fmul_rn(r, r);
        while (d > 0.0f && __fsqrt_rn(d) >= r) d = __int_as_float(__float_as_int(d) - 1);
        while (__fsqrt_rn(d) < r) d = __int_as_float(__float_as_int(d) + 1);
        thr[k] = d;
    }
    if (threadIdx.x == 0) thr[K] = __int_as_float(0x7f800000);  // no threshold past the last
    for (int k = threadIdx.x; k < 3 * L; k += blockDim.x) ls[k] = lights[k];
    for (int k = threadIdx.x; k < L; k += blockDim.x) wl[k] = lw ? lw[k] : 1.0f / (float)L;
    __syncthreads();
    // dtab[b] = #{k : thr_k < e_b}, e_b the float with bits AZ_TB0 + (b << AZ_SHIFT)
    for (int b = threadIdx.x; b < AZ_NB; b += blockDim.x) {
        const float eb = __int_as_float(AZ_TB0 + (b << AZ_SHIFT));
        int lo = 0, hi = K;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (thr[mid] < eb) lo = mid + 1; else hi = mid;
        }
        dtab[b] = (uint16_t)lo;
    }
    int several = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int bk = __float_as_int(thr[k]) - AZ_TB0;
        several |= bk < 0 || bk >= (AZ_NB << AZ_SHIFT);
        if (k + 1 < K) several |= (bk >> AZ_SHIFT) == ((__float_as_int(thr[k + 1]) - AZ_TB0) >> AZ_SHIFT);
    }
    const bool step_more = __syncthreads_or(several) != 0;
    const uint32_t plane = (uint32_t)H * (uint32_t)W;
    uint32_t phase = 0u;  // bit s: parity of the next wait on stage s
    bool failed = false;
    for (int j = 0; base < Q; base += nwarps * AZ_R, ++j) {
        const int cur = j & 1;
        float *sm = slice + cur * 3 * AZ_R;
        const int nr = (int)min((int64_t)AZ_R, Q - base);
        const int64_t nb = base + nwarps * AZ_R;
        if (lane == 0 && nb < Q && whole(nb)) {
            // the other stage: its bulk store (round j - 1) has read it out
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            az_issue(slice + (cur ^ 1) * 3 * AZ_R, qm, nb, bar0 + 8u * (cur ^ 1));
        }
        const bool w = whole(base);
        if (w) {
            const bool ok = az_wait(bar0 + 8u * cur, (phase >> cur) & 1u);
            phase ^= 1u << cur;
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0) {
                    record_status(status, DGSM_ERR_TIMEOUT);
                    // the copy issued for the next round is still in flight
                    if (nb < Q && whole(nb)) az_wait(bar0 + 8u * (cur ^ 1), (phase >> (cur ^ 1)) & 1u);
                }
                failed = true;
                break;
            }
        } else {
            // a bulk store of an earlier round may still read this stage
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            __syncwarp();
            for (int e = lane; e < 3 * nr; e += 32) sm[e] = qm[3 * base + e];
            __syncwarp();
        }
        float acc[AZ_U];
#pragma unroll
        for (int u = 0; u < AZ_U; ++u) acc[u] = 0.0f;
        for (int l = 0; l < L; ++l) {
            const float ox = ls[3 * l], oy = ls[3 * l + 1], oz = ls[3 * l + 2];
            const T *A = atlas + (size_t)l * K * plane;
            const T *Dy = DYN ? dyn + (size_t)l * K * plane : nullptr;
            float Tl[AZ_U];
            // receivers u = 2p, 2p + 1 as the two halves of packed f32x2
            // operations (each half rounded as the scalar operation)
#pragma unroll
            for (int p = 0; p < AZ_U / 2; ++p) {
                const int ra = 2 * p * 32 + lane, rb = ra + 32;
                const float2 M1 = make_float2(-1.0f, -1.0f);
                // x - o = fma(o, -1, x), rounded once
                const float2 vx = __ffma2_rn(make_float2(ox, ox), M1, make_float2(sm[3 * ra], sm[3 * rb]));
                const float2 vy = __ffma2_rn(make_float2(oy, oy), M1, make_float2(sm[3 * ra + 1], sm[3 * rb + 1]));
                const float2 vz = __ffma2_rn(make_float2(oz, oz), M1, make_float2(sm[3 * ra + 2], sm[3 * rb + 2]));
                const float2 d2 = __fadd2_rn(__fadd2_rn(__fmul2_rn(vx, vx), __fmul2_rn(vy, vy)), __fmul2_rn(vz, vz));
                // octahedral code (as xencode), both quotients by one rounded reciprocal
                const float2 sab = __fadd2_rn(__fadd2_rn(make_float2(fabsf(vx.x), fabsf(vx.y)),
                                                         make_float2(fabsf(vy.x), fabsf(vy.y))),
                                              make_float2(fabsf(vz.x), fabsf(vz.y)));
                const float2 y = make_float2(sab.x != 0.0f ? __frcp_rn(sab.x) : 0.0f,
                                             sab.y != 0.0f ? __frcp_rn(sab.y) : 0.0f);
                const float2 nsab = make_float2(-sab.x, -sab.y);
                const float2 q0x = __fmul2_rn(vx, y), q0y = __fmul2_rn(vy, y);
                float2 qx = __ffma2_rn(__ffma2_rn(nsab, q0x, vx), y, q0x);
                float2 qy = __ffma2_rn(__ffma2_rn(nsab, q0y, vy), y, q0y);
                if (sab.x < 1e-30f) {  // 1 / s near overflow (or s = 0): divide
                    qx.x = sab.x != 0.0f ? xdiv(vx.x, sab.x) : 0.0f;
                    qy.x = sab.x != 0.0f ? xdiv(vy.x, sab.x) : 0.0f;
                }
                if (sab.y < 1e-30f) {
                    qx.y = sab.y != 0.0f ? xdiv(vx.y, sab.y) : 0.0f;
                    qy.y = sab.y != 0.0f ? xdiv(vy.y, sab.y) : 0.0f;
                }
                float2 ux = qx, uy = qy;
                if (vz.x < 0.0f && sab.x != 0.0f) {
                    ux.x = xmul(sgn_pos(qx.x), xsub(1.0f, fabsf(qy.x)));
                    uy.x = xmul(sgn_pos(qy.x), xsub(1.0f, fabsf(qx.x)));
                }
                if (vz.y < 0.0f && sab.y != 0.0f) {
                    ux.y = xmul(sgn_pos(qx.y), xsub(1.0f, fabsf(qy.y)));
                    uy.y = xmul(sgn_pos(qy.y), xsub(1.0f, fabsf(qx.y)));
                }
                const float2 ONE = make_float2(1.0f, 1.0f), HALF = make_float2(0.5f, 0.5f),
                             NHALF = make_float2(-0.5f, -0.5f);
                const float2 gx = __fadd2_rn(__fmul2_rn(__fmul2_rn(__fadd2_rn(ux, ONE), HALF),
                                                        make_float2((float)W, (float)W)), NHALF);
                const float2 gy = __fadd2_rn(__fmul2_rn(__fmul2_rn(__fadd2_rn(uy, ONE), HALF),
                                                        make_float2((float)H, (float)H)), NHALF);
                const float2 bjf = make_float2(floorf(gx.x), floorf(gx.y));
                const float2 bif = make_float2(floorf(gy.x), floorf(gy.y));
                const float2 fxr = __ffma2_rn(bjf, M1, gx), fyr = __ffma2_rn(bif, M1, gy);
                float2 fx, fy, wt;
                uint32_t o[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float bjh = h ? bjf.y : bjf.x, bih = h ? bif.y : bif.x;
                    const int bj = (int)bjh, bi = (int)bih;
                    // taps (i0, i0 + 1) x (j0, j0 + 1); an edge by its weight (0 or 1)
                    const int j0 = min(max(bj, 0), W - 2), i0 = min(max(bi, 0), H - 2);
                    const float fxh = bj == j0 ? (h ? fxr.y : fxr.x) : (bj < j0 ? 0.0f : 1.0f);
                    const float fyh = bi == i0 ? (h ? fyr.y : fyr.x) : (bi < i0 ? 0.0f : 1.0f);
                    const float d2h = h ? d2.y : d2.x;
                    int k;  // #{r_k <= t}
                    if (!step_more) {
                        k = dtab[max(min((__float_as_int(d2h) - AZ_TB0) >> AZ_SHIFT, AZ_NB - 1), 0)];
                        k += thr[k] <= d2h ? 1 : 0;
                    } else {
                        k = 0;
                        while (k < K && thr[k] <= d2h) ++k;
                    }
                    // shells (k0, k0 + 1); below the first or past the last radius by the weight
                    const int k0 = min(max(k - 1, 0), K - 2);
                    const float wth =
                        k >= K ? 1.0f : fminf(fmaxf((d2h * rsqrtf(d2h) - rs[k0]) * inw[k0], 0.0f), 1.0f);
                    if (h) { fx.y = fxh; fy.y = fyh; wt.y = wth; }
                    else { fx.x = fxh; fy.x = fyh; wt.x = wth; }
                    o[h] = (uint32_t)k0 * plane + (uint32_t)i0 * W + (uint32_t)j0;
                }
                // lerp(a, b, f) = fma(f, b - a, a), both receivers at once
                auto lerp2 = [&](float2 a, float2 b, float2 f) { return __ffma2_rn(f, __ffma2_rn(a, M1, b), a); };
                auto bil2 = [&](const T *P0, const T *P1) {  // bilinear in the plane of one shell
                    const float2 a00 = make_float2(load_T(P0), load_T(P1));
                    const float2 a01 = make_float2(load_T(P0 + 1), load_T(P1 + 1));
                    const float2 a10 = make_float2(load_T(P0 + W), load_T(P1 + W));
                    const float2 a11 = make_float2(load_T(P0 + W + 1), load_T(P1 + W + 1));
                    return lerp2(lerp2(a00, a01, fx), lerp2(a10, a11, fx), fy);
                };
                auto tri2 = [&](const T *P) {
                    const T *pa = P + o[0], *pb = P + o[1];
                    return lerp2(bil2(pa, pb), bil2(pa + plane, pb + plane), wt);
                };
                float2 Tv = tri2(A);
                if (DYN) Tv = __fmul2_rn(Tv, tri2(Dy));
                Tl[2 * p] = d2.x != 0.0f ? Tv.x : 1.0f;
                Tl[2 * p + 1] = d2.y != 0.0f ? Tv.y : 1.0f;
            }
#pragma unroll
            for (int u = 0; u < AZ_U; ++u) {
                const int r = u * 32 + lane;
                if (HAS_T && r < nr) Tout[(base + r) * L + l] = Tl[u];
                acc[u] = fmaf(wl[l], Tl[u], acc[u]);
            }
        }
        // attenuated colours over the lane's own receivers' means, then out
#pragma unroll
        for (int u = 0; u < AZ_U; ++u) {
            const int r = u * 32 + lane;
            const float f = 1.0f - wd + wd * acc[u];
            const int64_t q = r < nr ? base + r : base;
            sm[3 * r] = __ldcs(cin + 3 * q) * f;
            sm[3 * r + 1] = __ldcs(cin + 3 * q + 1) * f;
            sm[3 * r + 2] = __ldcs(cin + 3 * q + 2) * f;
        }
        if (w) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                             ::"l"(cout + 3 * base), "r"(az_smem(sm)), "r"(AZ_BYTES) : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
        } else {
            __syncwarp();
            for (int e = lane; e < 3 * nr; e += 32) __stcs(cout + 3 * base + e, sm[e]);
        }
        __syncwarp();  // this stage is read before the next round's copy into it
    }
    (void)failed;
    // the bulk stores have finished before the block's shared memory goes
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---- footprint sampling (Sec. 3.3; ablation (A) of Sec. 4) ----------------

// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC 2011): ten rounds of two
// 64x64 -> 128-bit products, Weyl-sequence key schedule.
__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
    constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

constexpr int FP_THREADS = 128;
constexpr int FP_MAX_SAMPLES = 32;

// One receiver per thread.  Its sample points x_i = mu + R (s . z_i) are
// formed once in shared memory ([3 * n][FP_THREADS], conflict-free), then
// every light averages its lookups over them.
template <typename T>
__global__ void __launch_bounds__(FP_THREADS) attenuate_fp_kernel(
    const T *__restrict__ atlas, int L, int H, int W, const float *__restrict__ radii, int K,
    const float *__restrict__ lights, const float *__restrict__ qm, const float *__restrict__ qq,
    const float *__restrict__ qs, const float *cin, int64_t Q, const float *__restrict__ lw, float wd,
    int mode, int n_mc, uint64_t seed, float *cout, float *__restrict__ Tout) {
    extern __shared__ float pts[];
    __shared__ float rs[256], inw[256];
    __shared__ short tab[SHELL_BINS];
    __shared__ float ls[64 * 3];
    __shared__ float wl[64];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        rs[k] = radii[k];
        inw[k] = k + 1 < K ? 1.0f / (radii[k + 1] - radii[k]) : 0.0f;
    }
    for (int k = threadIdx.x; k < 3 * L; k += blockDim.x) ls[k] = lights[k];
    for (int k = threadIdx.x; k < L; k += blockDim.x) wl[k] = lw ? lw[k] : 1.0f / (float)L;
    __syncthreads();
    const ShellTab st = build_shell_tab(rs, K, tab);
    __syncthreads();
    const int n = mode == 0 ? 1 : mode == 1 ? 7 : n_mc;
    const float ea = 0.60653065971263342f;  // exp(-1/2)
    const float w_ctr = mode == 0 ? 1.0f : mode == 1 ? 1.0f / (1.0f + 6.0f * ea) : 1.0f / (float)n_mc;
    const float w_ax = mode == 1 ? ea / (1.0f + 6.0f * ea) : w_ctr;
    const int64_t lstride = (int64_t)K * H * W;
    float *px = pts + threadIdx.x;  // sample i coordinate c at px[(3 i + c) * FP_THREADS]
    for (int64_t q = (int64_t)blockIdx.x * FP_THREADS + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * FP_THREADS) {
        const float mx = __ldg(qm + 3 * q), my = __ldg(qm + 3 * q + 1), mz = __ldg(qm + 3 * q + 2);
        const float c0 = cin[3 * q], c1 = cin[3 * q + 1], c2 = cin[3 * q + 2];
        float R[9];
        {
            float w = __ldg(qq + 4 * q), x = __ldg(qq + 4 * q + 1), y = __ldg(qq + 4 * q + 2),
                  z = __ldg(qq + 4 * q + 3);
            const float inv = rsqrtf(w * w + x * x + y * y + z * z);
            w *= inv; x *= inv; y *= inv; z *= inv;
            R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
            R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
            R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
        }
        const float sc[3] = {__ldg(qs + 3 * q), __ldg(qs + 3 * q + 1), __ldg(qs + 3 * q + 2)};
        for (int i = 0; i < n; ++i) {
            px[(3 * i) * FP_THREADS] = mx;
            px[(3 * i + 1) * FP_THREADS] = my;
            px[(3 * i + 2) * FP_THREADS] = mz;
        }
        // offset component j (sample j / 3, axis j % 3) of size zj: x_i += R[:, c] s_c zj
        auto add = [&](int j, float zj) {
            const int i = j / 3, c = j - 3 * i;
            // column c of R and scale c by selects (no local-memory indexing)
            const float a = (c == 0 ? sc[0] : c == 1 ? sc[1] : sc[2]) * zj;
            const float r0 = c == 0 ? R[0] : c == 1 ? R[1] : R[2];
            const float r1 = c == 0 ? R[3] : c == 1 ? R[4] : R[5];
            const float r2 = c == 0 ? R[6] : c == 1 ? R[7] : R[8];
            px[(3 * i) * FP_THREADS] += r0 * a;
            px[(3 * i + 1) * FP_THREADS] += r1 * a;
            px[(3 * i + 2) * FP_THREADS] += r2 * a;
        };
        if (mode == 1) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                add(3 * (1 + 2 * a) + a, 1.0f);
                add(3 * (2 + 2 * a) + a, -1.0f);
            }
        } else if (mode == 2) {
            for (int b = 0; b * 8 < 3 * n; ++b) {
                uint64_t c[4] = {(uint64_t)q, (uint64_t)b, 0ull, 0ull};
                philox4x64(c, seed, 0ull);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const uint32_t lo = (uint32_t)c[p], hi = (uint32_t)(c[p] >> 32);
                    const float u1 = (float)((lo >> 8) + 1u) * 5.9604644775390625e-8f;
                    const float u2 = (float)((hi >> 8) + 1u) * 5.9604644775390625e-8f;
                    const float r = sqrtf(-2.0f * logf(u1));
                    float sn, cs;
                    sincospif(2.0f * u2, &sn, &cs);
                    const int j = 8 * b + 2 * p;
                    if (j < 3 * n) add(j, r * cs);
                    if (j + 1 < 3 * n) add(j + 1, r * sn);
                }
            }
        }
        float acc = 0.0f;
        for (int l = 0; l < L; ++l) {
            const float ox = ls[3 * l], oy = ls[3 * l + 1], oz = ls[3 * l + 2];
            const T *A = atlas + l * lstride;
            float Tl = 0.0f;
            for (int i = 0; i < n; ++i) {
                const SampleIndex s = sample_index_tab(px[(3 * i) * FP_THREADS], px[(3 * i + 1) * FP_THREADS],
                                                       px[(3 * i + 2) * FP_THREADS], ox, oy, oz, H, W, rs,
                                                       K, tab, st);
                const float Ti = s.t != 0.0f ? lookup(A, H, W, K, s, rs, inw) : 1.0f;
                Tl = fmaf(i == 0 ? w_ctr : w_ax, Ti, Tl);
            }
            if (Tout) Tout[q * L + l] = Tl;
            acc = fmaf(wl[l], Tl, acc);
        }
        const float f = 1.0f - wd + wd * acc;
        __stcs(cout + 3 * q, c0 * f);
        __stcs(cout + 3 * q + 1, c1 * f);
        __stcs(cout + 3 * q + 2, c2 * f);
    }
}

__global__ void sample_index_kernel(const float *__restrict__ pts, int64_t n,
                                    const float *__restrict__ light, int H, int W,
                                    const float *__restrict__ radii, int K,
                                    int32_t *__restrict__ idx_out, float *__restrict__ frac_out, int cube) {
    __shared__ float rs[256];
    __shared__ short tab[SHELL_BINS];
    for (int k = threadIdx.x; k < K; k += blockDim.x) rs[k] = radii[k];
    __syncthreads();
    const ShellTab st = build_shell_tab(rs, K, tab);
    __syncthreads();
    const float ox = light[0], oy = light[1], oz = light[2];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const SampleIndex s = cube ? sample_index_cube(pts[3 * q], pts[3 * q + 1], pts[3 * q + 2], ox, oy, oz, W,
                                                       rs, K, tab, st)
                                   : sample_index_tab(pts[3 * q], pts[3 * q + 1], pts[3 * q + 2], ox, oy, oz,
                                                      H, W, rs, K, tab, st);
        idx_out[5 * q] = s.ci;
        idx_out[5 * q + 1] = s.cj;
        idx_out[5 * q + 2] = s.bi;
        idx_out[5 * q + 3] = s.bj;
        idx_out[5 * q + 4] = s.k;
        frac_out[3 * q] = s.fy;
        frac_out[3 * q + 1] = s.fx;
        frac_out[3 * q + 2] = s.t;
    }
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

namespace {
// Resident blocks per SM of attenuate_stream_kernel<T, DYN, HAS_T> on device
// dev (its shared-memory limit raised first), found once per kernel and device.
template <typename T, bool DYN, bool HAS_T>
int az_blocks_per_sm(int dev) {
    auto kern = attenuate_stream_kernel<T, DYN, HAS_T>;
    static int cache[64] = {};  // blocks per SM + 1 per device (0: not yet found)
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev] - 1;
    int per_sm = 1;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AZ_SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, AZ_THREADS, AZ_SMEM);
    per_sm = std::max(per_sm, 1);
    if (dev >= 0 && dev < 64) cache[dev] = per_sm + 1;
    return per_sm;
}

template <typename T>
void launch_attenuate(int grid, cudaStream_t s, const void *atlas, const void *dyn, bool sep, int L,
                      int H, int W, const float *radii, int K, DynGeom dg, const float *lights,
                      const float *qm, const float *cin, int64_t Q, const float *lw, float wd,
                      float *cout, float *Tout, bool cube, int *status, int num_sms) {
    if (!cube && !sep && H >= 2 && W >= 2 && K >= 2) {
        // the streamed form: one resident wave of blocks
        const bool vec = ((((uintptr_t)qm) | ((uintptr_t)cin) | ((uintptr_t)cout)) & 15u) == 0;
        auto go = [&](auto kern, int per_sm) {
            const int64_t need = (Q + (int64_t)AZ_R * AZ_WARPS - 1) / ((int64_t)AZ_R * AZ_WARPS);
            const int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * per_sm));
            kern<<<g, AZ_THREADS, AZ_SMEM, s>>>((const T *)atlas, (const T *)dyn, L, H, W, radii, K, lights, qm,
                                                cin, Q, lw, wd, cout, Tout, vec, status);
        };
        int dev = 0;
        cudaGetDevice(&dev);
        if (dyn) {
            if (Tout) go(attenuate_stream_kernel<T, true, true>, az_blocks_per_sm<T, true, true>(dev));
            else go(attenuate_stream_kernel<T, true, false>, az_blocks_per_sm<T, true, false>(dev));
        } else {
            if (Tout) go(attenuate_stream_kernel<T, false, true>, az_blocks_per_sm<T, false, true>(dev));
            else go(attenuate_stream_kernel<T, false, false>, az_blocks_per_sm<T, false, false>(dev));
        }
        (void)grid;
        return;
    }
    if (cube)
        attenuate_kernel<T, false, true><<<grid, ATT_THREADS, 0, s>>>((const T *)atlas, nullptr, L, H, W,
            radii, K, dg, lights, qm, cin, Q, lw, wd, cout, Tout);
    else if (sep)
        attenuate_kernel<T, true><<<grid, ATT_THREADS, 0, s>>>((const T *)atlas, (const T *)dyn, L, H, W,
            radii, K, dg, lights, qm, cin, Q, lw, wd, cout, Tout);
    else
        attenuate_kernel<T, false><<<grid, ATT_THREADS, 0, s>>>((const T *)atlas, (const T *)dyn, L, H, W,
            radii, K, dg, lights, qm, cin, Q, lw, wd, cout, Tout);
}

int attenuate_common(dgsm_ctx *ctx, const void *atlas, const void *atlas_dyn, int32_t dtype,
                     int32_t L, int32_t H, int32_t W, const float *radii, int32_t K, bool sep,
                     DynGeom dg, const float *lights, const float *q_means,
                     const float *colors_in, int64_t n_q, const float *light_w,
                     float direct_frac, float *colors_out, float *T_out, void *stream, bool cube = false) {
    if (n_q < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "n_q < 0");
    if (L < 1 || L > 64) return fail(ctx, DGSM_ERR_INVALID_ARG, "need 1..64 lights");
    if (cube) {
        if (W < 1 || W > 4096 || H != 6 * W) return fail(ctx, DGSM_ERR_INVALID_ARG, "cube atlas: F in 1..4096");
    } else if (H < 1 || W < 1 || H > 4096 || W > 4096) {
        return fail(ctx, DGSM_ERR_INVALID_ARG, "H, W must be in 1..4096");
    }
    if (K < 1 || K > 256) return fail(ctx, DGSM_ERR_INVALID_ARG, "K must be in 1..256");
    if (sep && (dg.H < 1 || dg.W < 1 || dg.H > 4096 || dg.W > 4096 || dg.K < 1 || dg.K > 256 || !dg.radii))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "dynamic atlas: H, W in 1..4096, K in 1..256, radii required");
    if (dtype < DGSM_F32 || dtype > DGSM_BF16) return fail(ctx, DGSM_ERR_INVALID_ARG, "bad dtype");
    if (!atlas || !radii || !lights) return fail(ctx, DGSM_ERR_INVALID_ARG, "null atlas, radii or lights");
    if (n_q > 0 && (!q_means || !colors_in || !colors_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "null query array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n_q == 0) return DGSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t span = (int64_t)ATT_U * ATT_THREADS;
    const int grid = (int)std::min<int64_t>((n_q + span - 1) / span, (int64_t)ctx->num_sms * 8);
    switch (dtype) {
        case DGSM_F32:
            launch_attenuate<float>(grid, s, atlas, atlas_dyn, sep, L, H, W, radii, K, dg, lights, q_means,
                                    colors_in, n_q, light_w, direct_frac, colors_out, T_out, cube,
                                    ctx->d_status, ctx->num_sms);
            break;
        case DGSM_F16:
            launch_attenuate<__half>(grid, s, atlas, atlas_dyn, sep, L, H, W, radii, K, dg, lights, q_means,
                                     colors_in, n_q, light_w, direct_frac, colors_out, T_out, cube,
                                    ctx->d_status, ctx->num_sms);
            break;
        default:
            launch_attenuate<__nv_bfloat16>(grid, s, atlas, atlas_dyn, sep, L, H, W, radii, K, dg, lights,
                                            q_means, colors_in, n_q, light_w, direct_frac, colors_out, T_out,
                                            cube, ctx->d_status, ctx->num_sms);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "attenuate_kernel");
}
}  // namespace

extern "C" int dgsm_attenuate(dgsm_ctx *ctx, const void *atlas, const void *atlas_dyn,
                              int32_t dtype, int32_t L, int32_t H, int32_t W, const float *radii,
                              int32_t K, const float *lights, const float *q_means,
                              const float *colors_in, int64_t n_q, const float *light_w,
                              float direct_frac, float *colors_out, float *T_out, void *stream) {
    DGSM_RANGE("dgsm_attenuate");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    return attenuate_common(ctx, atlas, atlas_dyn, dtype, L, H, W, radii, K, false,
                            DynGeom{H, W, K, radii}, lights, q_means, colors_in, n_q, light_w,
                            direct_frac, colors_out, T_out, stream);
}

extern "C" int dgsm_attenuate_dyn(dgsm_ctx *ctx, const void *atlas, int32_t dtype, int32_t L,
                                  int32_t H, int32_t W, const float *radii, int32_t K,
                                  const void *atlas_dyn, int32_t H_dyn, int32_t W_dyn,
                                  const float *radii_dyn, int32_t K_dyn, const float *lights,
                                  const float *q_means, const float *colors_in, int64_t n_q,
                                  const float *light_w, float direct_frac, float *colors_out,
                                  float *T_out, void *stream) {
    DGSM_RANGE("dgsm_attenuate_dyn");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!atlas_dyn) return fail(ctx, DGSM_ERR_INVALID_ARG, "null dynamic atlas");
    return attenuate_common(ctx, atlas, atlas_dyn, dtype, L, H, W, radii, K, true,
                            DynGeom{H_dyn, W_dyn, K_dyn, radii_dyn}, lights, q_means, colors_in, n_q,
                            light_w, direct_frac, colors_out, T_out, stream);
}

extern "C" int dgsm_sample_index(dgsm_ctx *ctx, const float *points, int64_t n, const float *light,
                                 int32_t H, int32_t W, const float *radii, int32_t K,
                                 int32_t *idx_out, float *frac_out, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || H < 1 || W < 1 || H > 4096 || W > 4096 || K < 1 || K > 256)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "bad size");
    if (n > 0 && (!points || !light || !radii || !idx_out || !frac_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n == 0) return DGSM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
    sample_index_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(points, n, light, H, W, radii, K,
                                                                 idx_out, frac_out, 0);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "sample_index_kernel");
}

extern "C" int dgsm_attenuate_footprint(dgsm_ctx *ctx, const void *atlas, int32_t dtype, int32_t L,
                                        int32_t H, int32_t W, const float *radii, int32_t K,
                                        const float *lights, const float *q_means, const float *q_quats,
                                        const float *q_scales, const float *colors_in, int64_t n_q,
                                        const float *light_w, float direct_frac, int32_t mode,
                                        int32_t n_samples, uint64_t seed, float *colors_out, float *T_out,
                                        void *stream) {
    DGSM_RANGE("dgsm_attenuate_footprint");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n_q < 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "n_q < 0");
    if (L < 1 || L > 64) return fail(ctx, DGSM_ERR_INVALID_ARG, "need 1..64 lights");
    if (H < 1 || W < 1 || H > 4096 || W > 4096) return fail(ctx, DGSM_ERR_INVALID_ARG, "H, W must be in 1..4096");
    if (K < 1 || K > 256) return fail(ctx, DGSM_ERR_INVALID_ARG, "K must be in 1..256");
    if (dtype < DGSM_F32 || dtype > DGSM_BF16) return fail(ctx, DGSM_ERR_INVALID_ARG, "bad dtype");
    if (mode < DGSM_FP_CENTRE || mode > DGSM_FP_MC) return fail(ctx, DGSM_ERR_INVALID_ARG, "bad footprint mode");
    if (mode == DGSM_FP_MC && (n_samples < 1 || n_samples > FP_MAX_SAMPLES))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "n_samples must be in 1..32");
    if (!atlas || !radii || !lights) return fail(ctx, DGSM_ERR_INVALID_ARG, "null atlas, radii or lights");
    if (n_q > 0 && (!q_means || !q_quats || !q_scales || !colors_in || !colors_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "null query array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n_q == 0) return DGSM_OK;
    const int n = mode == DGSM_FP_CENTRE ? 1 : mode == DGSM_FP_STENCIL7 ? 7 : n_samples;
    const size_t smem = (size_t)3 * n * FP_THREADS * sizeof(float);
    const int grid = (int)std::min<int64_t>((n_q + FP_THREADS - 1) / FP_THREADS, (int64_t)ctx->num_sms * 16);
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype) {
        case DGSM_F32:
            e = cudaFuncSetAttribute(attenuate_fp_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                attenuate_fp_kernel<float><<<grid, FP_THREADS, smem, s>>>(
                    (const float *)atlas, L, H, W, radii, K, lights, q_means, q_quats, q_scales, colors_in, n_q,
                    light_w, direct_frac, mode, n_samples, seed, colors_out, T_out);
            break;
        case DGSM_F16:
            e = cudaFuncSetAttribute(attenuate_fp_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                attenuate_fp_kernel<__half><<<grid, FP_THREADS, smem, s>>>(
                    (const __half *)atlas, L, H, W, radii, K, lights, q_means, q_quats, q_scales, colors_in, n_q,
                    light_w, direct_frac, mode, n_samples, seed, colors_out, T_out);
            break;
        default:
            e = cudaFuncSetAttribute(attenuate_fp_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                attenuate_fp_kernel<__nv_bfloat16><<<grid, FP_THREADS, smem, s>>>(
                    (const __nv_bfloat16 *)atlas, L, H, W, radii, K, lights, q_means, q_quats, q_scales,
                    colors_in, n_q, light_w, direct_frac, mode, n_samples, seed, colors_out, T_out);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "attenuate_fp: smem attribute");
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "attenuate_fp_kernel");
}

extern "C" int dgsm_attenuate_cube(dgsm_ctx *ctx, const void *atlas, int32_t dtype, int32_t L, int32_t F,
                                   const float *radii, int32_t K, const float *lights, const float *q_means,
                                   const float *colors_in, int64_t n_q, const float *light_w, float direct_frac,
                                   float *colors_out, float *T_out, void *stream) {
    DGSM_RANGE("dgsm_attenuate_cube");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    return attenuate_common(ctx, atlas, nullptr, dtype, L, 6 * F, F, radii, K, false, DynGeom{6 * F, F, K, radii},
                            lights, q_means, colors_in, n_q, light_w, direct_frac, colors_out, T_out, stream, true);
}

extern "C" int dgsm_sample_index_cube(dgsm_ctx *ctx, const float *points, int64_t n, const float *light,
                                      int32_t F, const float *radii, int32_t K, int32_t *idx_out, float *frac_out,
                                      void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || F < 1 || F > 4096 || K < 1 || K > 256) return fail(ctx, DGSM_ERR_INVALID_ARG, "bad size");
    if (n > 0 && (!points || !light || !radii || !idx_out || !frac_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "null pointer");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n == 0) return DGSM_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
    sample_index_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(points, n, light, 6 * F, F, radii, K, idx_out,
                                                                 frac_out, 1);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "sample_index_kernel");
}
