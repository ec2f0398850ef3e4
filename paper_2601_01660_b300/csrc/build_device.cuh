// build_device.cuh -- device code of the atlas build (Sec. 3.2): record
// layouts, the direction cones and planes of atlas tiles, the per (light,
// Gaussian) prep, the cone and ellipsoid tests of the binning, one fine
// binning unit, and the tile worker that accumulates the closed form.  Used by
// build.cu's kernels and by the persistent frame kernel (frame_kernel.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {


constexpr int SUPER = 8;       // super-tile edge, in tiles
constexpr int REC_F4 = 4;      // float4 per build record
constexpr int BT_THREADS = 256;
constexpr int ITEM_CHUNKS = 16;  // a work item holds at most ITEM_CHUNKS * chunk Gaussians
#ifndef DGSM_BT_MIN_BLOCKS
#define DGSM_BT_MIN_BLOCKS 4        // resident build blocks per SM the register budget targets
#endif

// Per (light, Gaussian) record read by the build kernel (64 bytes):
//   r0 = (M00 M01 M02 M10), r1 = (M11 M12 M20 M21), r2 = (M22 w'x w'y w'z),
//   r3 = (beta sqrt(pi/2), k^2, packed window, 0)
// packed window: bits 0-9 first shell of the window, 10-19 first shell past
// it, bit 20 = light inside the Gaussian's culling sphere.
struct __align__(16) BuildRec {
    float4 r0, r1, r2, r3;
};

// Per (light, Gaussian) binning record (80 bytes): a = (dir xyz, cos theta),
// b = (sin theta, mode, k2s, v.x), c = (v.y, v.z, c0.x, c0.y),
// d = (c0.z, c1.x, c1.y, c1.z), e = (c2.x, c2.y, c2.z, -); mode 0 = not
// binned, 1 = cone and ellipsoid tests, 2 = all tiles.  v = mu - o, c_k =
// s_k times axis k of the Gaussian, k2s = k^2 (1 + 2^-10).
struct __align__(16) BinRec {
    float4 a, b, c, d, e;
};

// Gaussian index bits of a pair value; bits 30 and 31 hold the half-tile
// mask (bit 30: the top half of the tile may be hit, bit 31: the bottom).
constexpr uint32_t VAL_IDX = 0x3FFFFFFFu;
constexpr int PLANE_F4 = 5;  // float4 per tile: top, bottom, left, right, mid planes
constexpr unsigned FULLMASK = 0xffffffffu;

struct __align__(16) Item {
    uint32_t key, start, end, n_items;
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
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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

__device__ __forceinline__ float3 xcross(float3 a, float3 b) {
    return make_float3(xsub(xmul(a.y, b.z), xmul(a.z, b.y)), xsub(xmul(a.z, b.x), xmul(a.x, b.z)),
                       xsub(xmul(a.x, b.y), xmul(a.y, b.x)));
}

// Octahedral face of an atlas point: bit 0 u >= 0, bit 1 v >= 0, bit 2 the
// upper hemisphere (as xdecode decides it).
__device__ __forceinline__ int xface(float u, float v) {
    const float z = xsub(xsub(1.0f, fabsf(u)), fabsf(v));
    return (u >= 0.0f ? 1 : 0) | (v >= 0.0f ? 2 : 0) | (z >= 0.0f ? 4 : 0);
}

// Plane through the light containing directions a and b, non-negative on c's side.
__device__ __forceinline__ float3 xplane(float3 a, float3 b, float3 c) {
    float3 n = xcross(a, b);
    if (xdot(n.x, n.y, n.z, c.x, c.y, c.z) < 0.0f) n = make_float3(-n.x, -n.y, -n.z);
    return n;
}

// Separating planes of the texel-centre rectangle [j0,j1) x [i0,i1) for the
// ellipsoid test.  Inside one octahedral face the decode is affine in (u,v),
// so atlas lines are great circles and the rays through the rectangle's texel
// centres lie in the polyhedral cone of its corner directions.
// out[0] = (top edge plane, valid), out[1] = (bottom edge plane, has bottom
// half), out[2] = left, out[3] = right, out[4] = plane between the halves
// (rows [i0, i0+half) above, non-negative on their side).  valid = 0 when the
// rectangle spans two faces or is a single row or column (no plane test).
__device__ void rect_planes(int i0, int i1, int j0, int j1, int half, int H, int W, float4 *out) {
    const float ua = xcentre(j0, W), ub = xcentre(j1 - 1, W);
    const float va = xcentre(i0, H), vb = xcentre(i1 - 1, H);
    const float hb = i1 - i0 > half ? 1.0f : 0.0f;
    for (int q = 0; q < PLANE_F4; ++q) out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    out[1].w = hb;
    const int f = xface(ua, va);
    if (!(ua < ub && va < vb) || xface(ub, va) != f || xface(ua, vb) != f || xface(ub, vb) != f) return;
    const float uc = xmul(xadd(ua, ub), 0.5f), vc = xmul(xadd(va, vb), 0.5f);
    const float3 c = xdecode(uc, vc);
    const float3 d00 = xdecode(ua, va), d01 = xdecode(ub, va), d10 = xdecode(ua, vb), d11 = xdecode(ub, vb);
    const float3 top = xplane(d00, d01, c), bot = xplane(d10, d11, c);
    const float3 left = xplane(d00, d10, c), right = xplane(d01, d11, c);
    out[0] = make_float4(top.x, top.y, top.z, 1.0f);
    out[1] = make_float4(bot.x, bot.y, bot.z, hb);
    out[2] = make_float4(left.x, left.y, left.z, 0.0f);
    out[3] = make_float4(right.x, right.y, right.z, 0.0f);
    if (hb != 0.0f) {
        const float vm = xsub(xdiv((float)(2 * (i0 + half)), (float)H), 1.0f);
        const float3 mid = xplane(xdecode(ua, vm), xdecode(ub, vm), xdecode(uc, va));
        out[4] = make_float4(mid.x, mid.y, mid.z, 0.0f);
    }
}

// The ellipsoid test of a Gaussian (axes ax: v, c0, c1, c2) against one
// plane: does its culling ellipsoid reach the plane's non-negative side?
// Support n.v + k |(c_k . n)_k| compared in squares when n.v < 0.
struct GAxes {
    float v[3], c[9], k2s;
};

// Dot products of the plane tests as a fused chain a0 b0, then + a1 b1, then
// + a2 b2, each step one IEEE fused multiply-add (C's fmaf computes the same).
__device__ __forceinline__ float xfdot(float ax, float ay, float az, float bx, float by, float bz) {
    return __fmaf_rn(az, bz, __fmaf_rn(ay, by, __fmul_rn(ax, bx)));
}

__device__ __forceinline__ void plane_terms(const float4 &n, const GAxes &g, float &nv, float &reach) {
    nv = xfdot(n.x, n.y, n.z, g.v[0], g.v[1], g.v[2]);
    const float p0 = xfdot(n.x, n.y, n.z, g.c[0], g.c[1], g.c[2]);
    const float p1 = xfdot(n.x, n.y, n.z, g.c[3], g.c[4], g.c[5]);
    const float p2 = xfdot(n.x, n.y, n.z, g.c[6], g.c[7], g.c[8]);
    const float ss = xfdot(p0, p1, p2, p0, p1, p2);
    reach = (xmul(nv, nv) <= xmul(g.k2s, ss)) ? 1.0f : 0.0f;
}

__device__ __forceinline__ bool plane_ok(const float4 &n, const GAxes &g) {
    const float nv = xfdot(n.x, n.y, n.z, g.v[0], g.v[1], g.v[2]);
    if (nv >= 0.0f) return true;
    float nv2, reach;
    plane_terms(n, g, nv2, reach);
    return reach != 0.0f;
}

// Half-tile mask of a (Gaussian, tile) pair whose cones overlap: bit 0 the
// top half may be hit, bit 1 the bottom half; 0 = the tile is not reached.
__device__ __forceinline__ uint32_t half_mask(const float4 *pl, const GAxes &g, bool inside) {
    const float4 p1 = pl[1];
    const uint32_t hb = p1.w != 0.0f ? 2u : 0u;
    const float4 p0 = pl[0];
    if (inside || p0.w == 0.0f) return 1u | hb;
    if (!plane_ok(pl[2], g) || !plane_ok(pl[3], g)) return 0u;
    if (!hb) return plane_ok(p0, g) ? 1u : 0u;
    bool mid_pos = true, mid_neg = true;
    const float4 pm = pl[4];
    float nv, reach;
    plane_terms(pm, g, nv, reach);
    if (nv != 0.0f) {
        mid_pos = nv > 0.0f || reach != 0.0f;
        mid_neg = nv < 0.0f || reach != 0.0f;
    }
    uint32_t m = 0u;
    if (mid_pos && plane_ok(p0, g)) m |= 1u;
    if (mid_neg && plane_ok(p1, g)) m |= 2u;
    return m;
}

// The cone and planes of a texel-centre rectangle of a cube-map atlas
// (F x F faces stacked in rows; see xdecode_cube).  Inside a face the decode
// is a central projection of the face plane, so the rectangle's part on a
// face is a convex spherical quadrilateral (great-circle edges), and a cap of
// half-angle below 90 degrees (a convex set) holds it iff it holds its four
// corners.  The axis is the decoded centre for a rectangle on one face, the
// normalised sum of its parts' decoded centres for one across faces; the
// half-angle reaches the farthest corner of any part.
__device__ void rect_cone_cube(int i0, int i1, int j0, int j1, int F, float4 *out) {
    const int f0 = i0 / F, f1 = (i1 - 1) / F;
    const float ua = xcentre(j0, F), ub = xcentre(j1 - 1, F);
    const float uc = xmul(xadd(ua, ub), 0.5f);
    float3 c;
    if (f0 == f1) {
        const float va = xcentre(i0 - f0 * F, F), vb = xcentre(i1 - 1 - f0 * F, F);
        c = xdecode_cube(f0, uc, xmul(xadd(va, vb), 0.5f));
    } else {
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        for (int f = f0; f <= f1; ++f) {
            const float va = xcentre(max(i0, f * F) - f * F, F), vb = xcentre(min(i1, (f + 1) * F) - 1 - f * F, F);
            const float3 d = xdecode_cube(f, uc, xmul(xadd(va, vb), 0.5f));
            sx = xadd(sx, d.x);
            sy = xadd(sy, d.y);
            sz = xadd(sz, d.z);
        }
        const float n = xsqrt(xadd(xadd(xmul(sx, sx), xmul(sy, sy)), xmul(sz, sz)));
        if (!(n > 0.0f)) {
            out[0] = make_float4(0.0f, 0.0f, 1.0f, -1.0f);
            out[1] = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
            return;
        }
        c = make_float3(xdiv(sx, n), xdiv(sy, n), xdiv(sz, n));
    }
    float cmin = 1.0f;
    const float us[2] = {ua, ub};
    for (int f = f0; f <= f1; ++f) {
        const float vs[2] = {xcentre(max(i0, f * F) - f * F, F), xcentre(min(i1, (f + 1) * F) - 1 - f * F, F)};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float3 d = xdecode_cube(f, us[b], vs[a]);
                cmin = fminf(cmin, xdot(c.x, c.y, c.z, d.x, d.y, d.z));
            }
    }
    if (cmin <= 0.0f) {
        out[0] = make_float4(c.x, c.y, c.z, -1.0f);
        out[1] = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
    } else {
        out[0] = make_float4(c.x, c.y, c.z, cmin);
        out[1] = make_float4(xsqrt(xsub(1.0f, xmul(cmin, cmin))), 0.0f, 0.0f, 0.0f);
    }
}

__device__ void rect_planes_cube(int i0, int i1, int j0, int j1, int half, int F, float4 *out) {
    const int f = i0 / F;
    const float ua = xcentre(j0, F), ub = xcentre(j1 - 1, F);
    const float va = xcentre(i0 - f * F, F), vb = xcentre(i1 - 1 - f * F, F);
    const float hb = i1 - i0 > half ? 1.0f : 0.0f;
    for (int q = 0; q < PLANE_F4; ++q) out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    out[1].w = hb;
    if (!(ua < ub && va < vb) || (i1 - 1) / F != f) return;
    const float uc = xmul(xadd(ua, ub), 0.5f), vc = xmul(xadd(va, vb), 0.5f);
    const float3 c = xdecode_cube(f, uc, vc);
    const float3 d00 = xdecode_cube(f, ua, va), d01 = xdecode_cube(f, ub, va);
    const float3 d10 = xdecode_cube(f, ua, vb), d11 = xdecode_cube(f, ub, vb);
    const float3 top = xplane(d00, d01, c), bot = xplane(d10, d11, c);
    const float3 left = xplane(d00, d10, c), right = xplane(d01, d11, c);
    out[0] = make_float4(top.x, top.y, top.z, 1.0f);
    out[1] = make_float4(bot.x, bot.y, bot.z, hb);
    out[2] = make_float4(left.x, left.y, left.z, 0.0f);
    out[3] = make_float4(right.x, right.y, right.z, 0.0f);
    if (hb != 0.0f) {
        const float vm = xsub(xdiv((float)(2 * (i0 + half - f * F)), (float)F), 1.0f);
        const float3 mid = xplane(xdecode_cube(f, ua, vm), xdecode_cube(f, ub, vm), xdecode_cube(f, uc, va));
        out[4] = make_float4(mid.x, mid.y, mid.z, 0.0f);
    }
}

// cones: [0, n_tiles) tiles, then [n_tiles, n_tiles + n_super) super-tiles;
// two float4 per cone; then the tiles' planes, PLANE_F4 float4 each; then a
// second cone per super-tile.  On a cube map a super-tile across two faces
// (which lie anywhere on the sphere relative to each other: the faces are
// stacked in atlas rows) gets one cone per face part, the first flagged in
__device__ __forceinline__ void rect_cones_one(int idx, int H, int W, int tile, int tx, int ty, int sx, int sy,
                                               float4 *__restrict__ cones, int map) {
    const int n_tiles = tx * ty, n_super = sx * sy;
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
    float4 *second = idx >= n_tiles ? cones + 2 * (n_tiles + n_super) + PLANE_F4 * n_tiles + 2 * (idx - n_tiles)
                                    : nullptr;
    if (second) {
        second[0] = make_float4(0.0f, 0.0f, 1.0f, 2.0f);  // unused unless flagged
        second[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (map == MAP_CUBE) {
        const int i1 = min(i0 + edge, H), f0 = i0 / W, f1 = (i1 - 1) / W;
        if (second && f1 == f0 + 1) {
            rect_cone_cube(i0, f1 * W, j0, min(j0 + edge, W), W, cones + 2 * idx);
            rect_cone_cube(f1 * W, i1, j0, min(j0 + edge, W), W, second);
            cones[2 * idx + 1].z = 1.0f;
            return;
        }
        rect_cone_cube(i0, i1, j0, min(j0 + edge, W), W, cones + 2 * idx);
        if (idx < n_tiles)
            rect_planes_cube(i0, min(i0 + edge, H), j0, min(j0 + edge, W), tile / 2, W,
                             cones + 2 * (n_tiles + n_super) + PLANE_F4 * idx);
        return;
    }
    rect_cone(i0, min(i0 + edge, H), j0, min(j0 + edge, W), H, W, cones + 2 * idx);
    if (idx < n_tiles)
        rect_planes(i0, min(i0 + edge, H), j0, min(j0 + edge, W), tile / 2, H, W,
                    cones + 2 * (n_tiles + n_super) + PLANE_F4 * idx);
}

// ---------------------------------------------------------------------------
// Per (light, Gaussian) preparation.
// ---------------------------------------------------------------------------
// One (light l, Gaussian g) of the prep, idx = l N + g, from the Gaussian's
// mean, scales, rotation (w, x, y, z) and opacity and the light's position:
// its binning record (bin_out) and (brec != nullptr) its build record
// brec[idx].
__device__ __forceinline__ void prep_core(
    int64_t idx, int l, float mx, float my, float mz, float s0, float s1, float s2, float qw, float qx,
    float qy, float qz, float alpha, float ox, float oy, float oz, const float *__restrict__ radii, int K,
    float kappa, float eps, BuildRec *__restrict__ brec, BinRec &bin_out, int *__restrict__ status,
    const int *__restrict__ roi_k, int beta_mode) {
    BinRec br;
    br.a = make_float4(0.f, 0.f, 1.f, -1.f);
    br.b = make_float4(0.f, 0.f, 0.f, 0.f);  // mode 0: not binned
    br.c = br.d = br.e = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(s0) &&
                        isfinite(s1) && isfinite(s2) && isfinite(qw) && isfinite(qx) &&
                        isfinite(qy) && isfinite(qz) && isfinite(alpha) && s0 > 0.f &&
                        s1 > 0.f && s2 > 0.f;
    if (!finite) {
        record_status(status, DGSM_ERR_NONFINITE_INPUT);
        bin_out = br;
        return;
    }
    // --- binning specification (IEEE single ops, bit-exact with the CPU) ---
    float a = alpha;
    if (!(a > 0.0f)) {
        bin_out = br;
        return;
    }
    a = fminf(a, 0.999999f);
    const float smax = fmaxf(fmaxf(s0, s1), s2);
    const float smin = fminf(fminf(s0, s1), s2);
    const float odds = xdiv(a, xsub(1.0f, a));
    // bound of beta sqrt(2 pi / a) / tau* along any ray, per mapping
    float gbound;
    if (beta_mode == 1) gbound = xmul(2.50662827f, smax);
    else if (beta_mode == 3) gbound = xdiv(smax, xmul(6.28318531f, xmul(xmul(s0, s1), s2)));
    else gbound = xdiv(smax, smin);
    const float Q = xdiv(xmul(xmul(kappa, odds), gbound), eps);
    int e = 0;
    frexpf(Q, &e);
    e = max(e, 1);
    const float k2 = xmul(1.38629436f, (float)e);
    const float r = xmul(xsqrt(k2), smax);
    const float vx = xsub(mx, ox), vy = xsub(my, oy), vz = xsub(mz, oz);
    const float dist = xsqrt(xadd(xadd(xmul(vx, vx), xmul(vy, vy)), xmul(vz, vz)));
    const float lo = xsub(dist, r);
    const int klast = roi_k ? roi_k[2 * l + 1] : K - 1;
    if (klast < 0 || lo > radii[klast]) {
        bin_out = br;
        return;
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
    {
        // axes of the culling ellipsoid (binning specification, exact ops)
        const float n = xsqrt(xadd(xadd(xadd(xmul(qw, qw), xmul(qx, qx)), xmul(qy, qy)), xmul(qz, qz)));
        const float w = xdiv(qw, n), x = xdiv(qx, n), y = xdiv(qy, n), z = xdiv(qz, n);
        const float pxx = xmul(x, x), pyy = xmul(y, y), pzz = xmul(z, z);
        const float pxy = xmul(x, y), pxz = xmul(x, z), pyz = xmul(y, z);
        const float pwx = xmul(w, x), pwy = xmul(w, y), pwz = xmul(w, z);
        const float r00 = xsub(1.0f, xmul(2.0f, xadd(pyy, pzz)));
        const float r11 = xsub(1.0f, xmul(2.0f, xadd(pxx, pzz)));
        const float r22 = xsub(1.0f, xmul(2.0f, xadd(pxx, pyy)));
        const float r01 = xmul(2.0f, xsub(pxy, pwz)), r10 = xmul(2.0f, xadd(pxy, pwz));
        const float r02 = xmul(2.0f, xadd(pxz, pwy)), r20 = xmul(2.0f, xsub(pxz, pwy));
        const float r12 = xmul(2.0f, xsub(pyz, pwx)), r21 = xmul(2.0f, xadd(pyz, pwx));
        br.b.z = xmul(k2, 1.0009765625f);
        br.b.w = vx;
        br.c = make_float4(vy, vz, xmul(r00, s0), xmul(r10, s0));
        br.d = make_float4(xmul(r20, s0), xmul(r01, s1), xmul(r11, s1), xmul(r21, s1));
        br.e = make_float4(xmul(r02, s2), xmul(r12, s2), xmul(r22, s2), 0.f);
    }
    bin_out = br;
    if (!brec) return;

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
    // beta sqrt(pi/2), beta from the opacity-to-absorption mapping:
    //   1: kappa tau*;  2 (Eq. 5): kappa tau* sqrt(tr A / 3) / sqrt(2 pi);
    //   3: kappa tau* / ((2 pi)^(3/2) s0 s1 s2)
    float bpref;
    if (beta_mode == 1) bpref = 1.25331414f * kappa * tau_star;
    else if (beta_mode == 3) bpref = 1.25331414f * kappa * tau_star / (15.7496099f * (s0 * s1 * s2));
    else bpref = 0.5f * kappa * tau_star * sqrtf(trA * (1.0f / 3.0f));
    const float hi = dist + r;
    int klo = 0, kend = 0;
    if (!inside) {
        while (klo < K && radii[klo] < lo) ++klo;
    }
    kend = klo;
    while (kend < K && radii[kend] <= hi) ++kend;
    const int packed = klo | (kend << 10) | ((inside ? 1 : 0) << 20);
    BuildRec rec;
    rec.r0 = make_float4(M00, M01, M02, M10);
    rec.r1 = make_float4(M11, M12, M20, M21);
    rec.r2 = make_float4(M22, wx, wy, wz);
    rec.r3 = make_float4(bpref, k2, __int_as_float(packed), 0.f);
    brec[idx] = rec;
}

// The same, reading Gaussian g and light l from their arrays.
__device__ __forceinline__ void prep_one(
    int64_t idx, int l, int64_t g, const float *__restrict__ means, const float *__restrict__ scales,
    const float *__restrict__ quats, const float *__restrict__ opac, const float *__restrict__ lights,
    const float *__restrict__ radii, int K, float kappa, float eps, BuildRec *__restrict__ brec,
    BinRec &bin_out, int *__restrict__ status, const int *__restrict__ roi_k, int beta_mode) {
    prep_core(idx, l, means[3 * g], means[3 * g + 1], means[3 * g + 2], scales[3 * g], scales[3 * g + 1],
              scales[3 * g + 2], quats[4 * g], quats[4 * g + 1], quats[4 * g + 2], quats[4 * g + 3], opac[g],
              lights[3 * l], lights[3 * l + 1], lights[3 * l + 2], radii, K, kappa, eps, brec, bin_out, status,
              roi_k, beta_mode);
}

__device__ __forceinline__ bool cone_overlap_v(const BinRec &g, const float4 &c0, const float4 &c1) {
    if (c1.y != 0.0f) return true;  // cone spans a hemisphere
    const float dot = xdot(g.a.x, g.a.y, g.a.z, c0.x, c0.y, c0.z);
    const float rhs = xsub(xmul(g.a.w, c0.w), xmul(g.b.x, c1.x));
    return dot >= rhs;
}

// cone: two float4 in global memory
__device__ __forceinline__ bool cone_overlap(const BinRec &g, const float4 *cone) {
    return cone_overlap_v(g, __ldg(cone), __ldg(cone + 1));
}

// Super-tile sidx of a cube map: its cone, or either of its two cones when
// flagged (the octahedral map's super-tiles have one cone).
__device__ __forceinline__ bool super_overlap(const BinRec &g, const float4 *scones, const float4 *scones2,
                                              int sidx) {
    const float4 c0 = __ldg(scones + 2 * sidx), c1 = __ldg(scones + 2 * sidx + 1);
    if (cone_overlap_v(g, c0, c1)) return true;
    return c1.z != 0.0f && cone_overlap(g, scones2 + 2 * sidx);
}

// ---------------------------------------------------------------------------
// Binning in two levels.  Pass A (Gaussian-major): each (light, Gaussian)
// tests its bounding cone against the cones of the 8x8-tile super-tiles and
// emits (light * n_super + super-tile, Gaussian) pairs; a stable sort by key
// gives every super-tile its Gaussian list in index order.  Pass B
// (super-tile-major): a block takes up to UNIT_G Gaussians of one list, stages
// the super-tile's 64 tile cones and planes and the Gaussians' records in
// shared memory, and each warp tests its 8 tiles (cone test, then the
// ellipsoid test on consecutive lanes); per-tile lists come out in Gaussian
// order, laid out super-tile by super-tile, with no sort.
// ---------------------------------------------------------------------------
constexpr int UNIT_G = 512;     // Gaussians of one super-tile list per fine-binning block
constexpr int FB_STAGE = 256;   // Gaussians staged in shared memory at a time
constexpr int TDAT_F4 = 2 + PLANE_F4;  // per tile: cone (2 float4) + planes

// unit = (super key, list start, list end, index within the key | units of the key << 16, first unit of the key)
struct __align__(16) Unit {
    uint32_t key, start, end, ju, u0, pad0, pad1, pad2;
};


// Pass B, count: per (unit, tile) the pair count into fcnt and three bitmaps
// over the unit's Gaussians (reaches the tile, its top half, its bottom half)
// into fmask, UNIT_G / 32 words each.  Entry of (tile t of super key k, unit j
// of U) in fcnt/foff: 64 u0 + t U + j, so that the scan lays out each tile's
// pairs unit after unit, i.e. in Gaussian order.
constexpr int MASK_WORDS = UNIT_G / 32;

// Shared memory of one fine-binning unit (FINE_SMEM_BYTES, carved by the caller).
constexpr int FB_WARPS = 8;                 // warps of a fine-binning block (256 threads)
constexpr int FB_PAIRS = 32 * 16;           // (Gaussian, quad) pairs a warp can hold: 16 quads per lane
struct FineSmem {
    float4 *tdat;           // [64 * TDAT_F4] the super-tile's tile cones and planes
    float4 *qc;             // [16 * 2] cones of its 2x2-tile quads (see quad_cones)
    BinRec *grec;           // [FB_STAGE] the staged Gaussians' records
    uint32_t *running;      // [64] pairs found per tile
    int *tvalid;            // [64] tile exists (and is active)
    uint32_t (*wm)[64][3];  // [FB_WARPS][64][3] each warp's word of bitmaps per tile; zero on entry and exit
    uint16_t (*plist)[FB_PAIRS];  // [FB_WARPS][FB_PAIRS] each warp's (lane << 4 | quad) pairs
    uint16_t (*plist2)[128];      // [FB_WARPS][128] each warp's (lane << 6 | tile) pairs of 32 quad pairs
};
constexpr size_t FINE_SMEM_BYTES = sizeof(float4) * (64 * TDAT_F4 + 32) + sizeof(BinRec) * FB_STAGE +
                                   sizeof(uint32_t) * 64 + sizeof(int) * 64 +
                                   sizeof(uint32_t) * FB_WARPS * 64 * 3 + sizeof(uint16_t) * FB_WARPS * (FB_PAIRS + 128);

__device__ __forceinline__ FineSmem fine_smem(void *base) {
    FineSmem sm;
    char *p = (char *)base;
    sm.tdat = (float4 *)p; p += sizeof(float4) * 64 * TDAT_F4;
    sm.qc = (float4 *)p; p += sizeof(float4) * 32;
    sm.grec = (BinRec *)p; p += sizeof(BinRec) * FB_STAGE;
    sm.running = (uint32_t *)p; p += sizeof(uint32_t) * 64;
    sm.tvalid = (int *)p; p += sizeof(int) * 64;
    sm.wm = (uint32_t(*)[64][3])p; p += sizeof(uint32_t) * FB_WARPS * 64 * 3;
    sm.plist = (uint16_t(*)[FB_PAIRS])p; p += sizeof(uint16_t) * FB_WARPS * FB_PAIRS;
    sm.plist2 = (uint16_t(*)[128])p;
    return sm;
}

// Quad q (tiles rows 2 (q / 4) + {0, 1}, columns 2 (q % 4) + {0, 1} of the
// super-tile): a cone holding the cones of its valid tiles, as (axis xyz,
// cos phi), (sin phi, flag, -, -), flag 0 = no valid tile, 1 = a cone,
// 2 = every direction.  Axis c = the normalised sum of the tile axes, phi =
// max over the tiles of (angle(c, axis_t) + phi_t) + 3e-3 rad; by the
// triangle inequality on the sphere, a Gaussian cone that overlaps a tile's
// cone then overlaps the quad's, and the 3e-3 rad and the 1e-5 slack of
// quad_overlap cover the rounding of both tests (a cosine compared within
// 1e-6 moves the angle by at most sqrt(2e-6) < 1.5e-3 rad).  A quad of
// half-angle beyond pi/2 - 3e-3 (or holding a whole-sphere tile) admits every
// Gaussian, whose cone is narrower than pi/2.
__device__ __forceinline__ void quad_cone(const float4 *tdat, const int *tvalid, int q, float4 *out) {
    const int t0 = (2 * (q / 4)) * SUPER + 2 * (q % 4);
    float cx = 0.f, cy = 0.f, cz = 0.f;
    bool any = false, whole = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int t = t0 + (k >> 1) * SUPER + (k & 1);
        if (!tvalid[t]) continue;
        const float4 c0 = tdat[TDAT_F4 * t], c1 = tdat[TDAT_F4 * t + 1];
        any = true;
        whole |= c1.y != 0.0f;
        cx += c0.x; cy += c0.y; cz += c0.z;
    }
    if (!any) {
        out[0] = make_float4(0.f, 0.f, 1.f, 1.f);
        out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float cn = sqrtf(cx * cx + cy * cy + cz * cz);
    float phi = 0.0f;
    if (!whole && cn > 1e-6f) {
        cx /= cn; cy /= cn; cz /= cn;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = t0 + (k >> 1) * SUPER + (k & 1);
            if (!tvalid[t]) continue;
            const float4 c0 = tdat[TDAT_F4 * t], c1 = tdat[TDAT_F4 * t + 1];
            const float d = fminf(fmaxf(cx * c0.x + cy * c0.y + cz * c0.z, -1.0f), 1.0f);
            phi = fmaxf(phi, acosf(d) + atan2f(c1.x, c0.w));
        }
        phi += 3e-3f;
    }
    if (whole || cn <= 1e-6f || phi >= 1.5707963f - 3e-3f) {
        out[0] = make_float4(0.f, 0.f, 1.f, -1.f);
        out[1] = make_float4(1.f, 2.f, 0.f, 0.f);
        return;
    }
    out[0] = make_float4(cx, cy, cz, cosf(phi));
    out[1] = make_float4(sinf(phi), 1.f, 0.f, 0.f);
}

// Does Gaussian cone g (axis g.a.xyz, cos g.a.w, sin g.b.x) reach quad cone
// (c0, c1)?  Looser than the tiles' exact test (see quad_cone).
__device__ __forceinline__ bool quad_overlap(const BinRec &g, const float4 &c0, const float4 &c1) {
    if (c1.y == 0.0f) return false;
    if (c1.y == 2.0f) return true;
    const float dot = fmaf(g.a.x, c0.x, fmaf(g.a.y, c0.y, g.a.z * c0.z));
    return dot >= fmaf(g.a.w, c0.w, -g.b.x * c1.x) - 1e-5f;
}

// Fine binning of unit u (all threads of the block): each warp takes 32 of
// its Gaussians at a time; a Gaussian's cone is tested against the 16 quad
// cones, the passing (Gaussian, quad) pairs are spread over the lanes, and
// each pair gets the exact tests of the quad's tiles (the cone test, then
// the ellipsoid planes).  Writes the unit's three bitmaps per tile to fmask
// (the same bits as testing every tile: the quad test only skips tiles whose
// exact cone test fails) and leaves the per-tile pair counts in sm.running
// (read them after this returns; the call ends with a barrier).  tact (or
// nullptr): per (light, tile) 1 if it holds a texel of the region of
// interest.
// rec(l, g) gives the binning record of Gaussian g for light l (read from the
// prep's records, or formed anew).
template <typename RecF>
__device__ __forceinline__ void fine_count_unit(const Unit &U, unsigned long long u,
                                                const uint32_t *__restrict__ cvals, RecF rec, int tx, int ty,
                                                int sx, int n_tiles, int n_super, const float4 *__restrict__ cones,
                                                uint32_t *__restrict__ fmask, const uint8_t *__restrict__ tact,
                                                const FineSmem &sm) {
    const float4 *planes = cones + 2 * (n_tiles + n_super);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int l = (int)(U.key / (uint32_t)n_super), sidx = (int)(U.key - (uint32_t)l * n_super);
    const int sa = sidx / sx, sb = sidx - sa * sx;
    __syncthreads();  // shared state of the previous unit is no longer read
    for (int e = tid; e < 64 * TDAT_F4; e += blockDim.x) {
        const int t = e / TDAT_F4, part = e - t * TDAT_F4;
        const int a = sa * SUPER + t / SUPER, b = sb * SUPER + t % SUPER;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a < ty && b < tx) {
            const int gt = a * tx + b;
            v = part < 2 ? __ldg(cones + 2 * gt + part) : __ldg(planes + PLANE_F4 * gt + part - 2);
        }
        sm.tdat[e] = v;
    }
    if (tid < 64) {
        const int a = sa * SUPER + tid / SUPER, b = sb * SUPER + tid % SUPER;
        sm.tvalid[tid] = a < ty && b < tx && (!tact || tact[l * n_tiles + a * tx + b]);
        sm.running[tid] = 0u;
    }
    __syncthreads();
    if (tid < 16) quad_cone(sm.tdat, sm.tvalid, tid, sm.qc + 2 * tid);
    __syncthreads();  // the quad cones are ready
    uint32_t *um = fmask + (size_t)u * 64 * 3 * MASK_WORDS;
    uint32_t (*wm)[3] = sm.wm[warp];
    uint16_t *pl = sm.plist[warp], *pl2 = sm.plist2[warp];
    BinRec *wrec = sm.grec + warp * 32;  // this warp's 32 staged records
    const int ng = (int)(U.end - U.start);
    // warp w takes the unit's groups of 32 Gaussians w, w + 8, ... and stages
    // its own records: no block barrier until the unit is done
    for (int grp = warp * 32; grp < ng; grp += FB_WARPS * 32) {
        const int word = grp / 32;
        const int gl = grp + lane;
        const bool gv = gl < ng;
        __syncwarp();  // the previous group's records are no longer read
        // the lane keeps its own record's cone (G.a, G.b) in registers; the
        // others read the staged copy
        BinRec G;
        G.a = make_float4(0.f, 0.f, 1.f, -1.f);
        G.b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gv) {
            const BinRec R = rec(l, cvals[U.start + gl]);
            wrec[lane] = R;
            G.a = R.a;
            G.b = R.b;
        }
        __syncwarp();
        const bool inside = G.b.y == 2.0f;
        // quads this Gaussian may reach
        uint32_t qm = 0u;
        if (gv && G.b.y != 0.0f) {
#pragma unroll 4
            for (int q = 0; q < 16; ++q) {
                const float4 c0 = sm.qc[2 * q], c1 = sm.qc[2 * q + 1];
                if (c1.y != 0.0f && (inside || quad_overlap(G, c0, c1))) qm |= 1u << q;
            }
        }
        // spread the (Gaussian, quad) pairs over the warp's list
        const int cnt = __popc(qm);
        int off = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULLMASK, off, o);
            if (lane >= o) off += y;
        }
        const int total = __shfl_sync(FULLMASK, off, 31);
        off -= cnt;
        for (uint32_t m = qm; m; m &= m - 1) pl[off++] = (uint16_t)((lane << 4) | (__ffs(m) - 1));
        __syncwarp();
        for (int r = 0; r < total; r += 32) {
            // the cone tests of the quads' tiles, one (Gaussian, quad) pair per lane ...
            const int e = r + lane;
            uint32_t tm = 0u;
            int gln = 0, t0 = 0;
            if (e < total) {
                const int pq = pl[e], q = pq & 15;
                gln = pq >> 4;
                t0 = (2 * (q / 4)) * SUPER + 2 * (q % 4);
                BinRec Rc;
                Rc.a = wrec[gln].a;
                Rc.b = wrec[gln].b;
                const bool rin = Rc.b.y == 2.0f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int t = t0 + (k >> 1) * SUPER + (k & 1);
                    if (sm.tvalid[t] && (rin || cone_overlap_v(Rc, sm.tdat[TDAT_F4 * t], sm.tdat[TDAT_F4 * t + 1])))
                        tm |= 1u << k;
                }
            }
            // ... then the ellipsoid tests of the passing (Gaussian, tile) pairs on consecutive lanes
            const int c2 = __popc(tm);
            int o2 = c2;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULLMASK, o2, o);
                if (lane >= o) o2 += y;
            }
            const int total2 = __shfl_sync(FULLMASK, o2, 31);
            o2 -= c2;
            for (uint32_t m = tm; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                pl2[o2++] = (uint16_t)((gln << 6) | (t0 + (k >> 1) * SUPER + (k & 1)));
            }
            __syncwarp();
            for (int r2 = 0; r2 < total2; r2 += 32) {
                const int e2 = r2 + lane;
                if (e2 < total2) {
                    const int v = pl2[e2], g2 = v >> 6, t = v & 63;
                    const BinRec &R = wrec[g2];
                    uint32_t hm;
                    if (R.b.y == 2.0f) {
                        hm = sm.tdat[TDAT_F4 * t + 3].w != 0.0f ? 3u : 1u;
                    } else {
                        GAxes ax;
                        ax.v[0] = R.b.w; ax.v[1] = R.c.x; ax.v[2] = R.c.y;
                        ax.c[0] = R.c.z; ax.c[1] = R.c.w; ax.c[2] = R.d.x;
                        ax.c[3] = R.d.y; ax.c[4] = R.d.z; ax.c[5] = R.d.w;
                        ax.c[6] = R.e.x; ax.c[7] = R.e.y; ax.c[8] = R.e.z;
                        ax.k2s = R.b.z;
                        hm = half_mask(sm.tdat + TDAT_F4 * t + 2, ax, false);
                    }
                    const uint32_t bit = 1u << g2;
                    if (hm) atomicOr(&wm[t][0], bit);
                    if (hm & 1u) atomicOr(&wm[t][1], bit);
                    if (hm & 2u) atomicOr(&wm[t][2], bit);
                }
            }
            __syncwarp();
        }
        __syncwarp();
        // this warp's word of every tile's bitmaps, then cleared
        for (int t = lane; t < 64; t += 32) {
            const uint32_t p = wm[t][0];
            if (p) atomicAdd(&sm.running[t], (uint32_t)__popc(p));
        }
        for (int k = lane; k < 64 * 3; k += 32) {
            const int t = k / 3, m = k - 3 * t;
            um[(t * 3 + m) * MASK_WORDS + word] = wm[t][m];
            wm[t][m] = 0u;
        }
        __syncwarp();
    }
    __syncthreads();
}

// Writes the pairs of tile t from one fine-binning unit's bitmaps um (its
// ng Gaussians' indices in gidx, shared memory) at vals[pos0 ...] in Gaussian
// order, each index with its half-tile mask (and keys[...] = key when keys
// != nullptr); positions at or past cap are skipped.  One warp: lane w loads
// word w of the three bitmaps (all the tile's words in flight together).
// When many words hold pairs, pair i of the tile goes to lane i % 32, which
// finds its word by a binary search over the words' running counts
// (shuffles) and its bit with __fns, so that every round writes 32
// consecutive pairs; when few do, the words are taken one at a time.
__device__ __forceinline__ void emit_tile(const uint32_t *__restrict__ um, int t, int ng, uint32_t pos0,
                                          const uint32_t *gidx, uint32_t *__restrict__ vals,
                                          uint32_t *__restrict__ keys, uint32_t key, uint32_t cap) {
    const int lane = threadIdx.x & 31;
    const int nw = (ng + 31) / 32;
    uint32_t p = 0u, tt = 0u, bb = 0u;
    if (lane < nw) {
        p = um[(t * 3 + 0) * MASK_WORDS + lane];
        tt = um[(t * 3 + 1) * MASK_WORDS + lane];
        bb = um[(t * 3 + 2) * MASK_WORDS + lane];
    }
    const int c = __popc(p);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULLMASK, incl, 31);
    const int excl = incl - c;
    const unsigned nz = __ballot_sync(FULLMASK, p != 0u);
    if (__popc(nz) <= 2 * ((total + 31) >> 5)) {
        // few words hold pairs: one word at a time, its pairs on their lanes
        const unsigned lt = (1u << lane) - 1u;
        for (unsigned m = nz; m; m &= m - 1) {
            const int w = __ffs(m) - 1;
            const uint32_t pw = __shfl_sync(FULLMASK, p, w), tw = __shfl_sync(FULLMASK, tt, w);
            const uint32_t bw = __shfl_sync(FULLMASK, bb, w);
            const int ew = __shfl_sync(FULLMASK, excl, w);
            if ((pw >> lane) & 1u) {
                const uint32_t hm = ((tw >> lane) & 1u) | (((bw >> lane) & 1u) << 1);
                const uint32_t pos = pos0 + (uint32_t)ew + __popc(pw & lt);
                if (pos < cap) {
                    vals[pos] = gidx[32 * w + lane] | (hm << 30);
                    if (keys) keys[pos] = key;
                }
            }
        }
        return;
    }
    for (int r0 = 0; r0 < total; r0 += 32) {
        const int i = r0 + lane;
        // w = the first word whose running count passes i
        int w = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int v = __shfl_sync(FULLMASK, incl, w + step - 1);
            if (v <= i) w += step;
        }
        w = min(w, 31);
        const uint32_t pw = __shfl_sync(FULLMASK, p, w), tw = __shfl_sync(FULLMASK, tt, w);
        const uint32_t bw = __shfl_sync(FULLMASK, bb, w);
        const int ew = __shfl_sync(FULLMASK, excl, w);
        if (i < total) {
            const int bit = (int)__fns(pw, 0u, i - ew + 1);
            const uint32_t hm = ((tw >> bit) & 1u) | (((bw >> bit) & 1u) << 1);
            const uint32_t pos = pos0 + (uint32_t)i;
            if (pos < cap) {
                vals[pos] = gidx[32 * w + bit] | (hm << 30);
                if (keys) keys[pos] = key;
            }
        }
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

// Geometry of one (texel ray, Gaussian) pair in the Gaussian's whitened
// frame: d' = M d, a = |d'|^2 = d^T A d, pw = d'.w' = -b, c2 = |w' x d'|^2 =
// m^2 a (the Lagrange identity: no cancellation of large squares).
struct PairGeom {
    float a, pw, c2;
};

__device__ __forceinline__ PairGeom pair_geom(const float4 &q0, const float4 &q1, const float4 &q2,
                                              float dx, float dy, float dz) {
    const float px = fmaf(q0.x, dx, fmaf(q0.y, dy, q0.z * dz));
    const float py = fmaf(q0.w, dx, fmaf(q1.x, dy, q1.y * dz));
    const float pz = fmaf(q1.z, dx, fmaf(q1.w, dy, q2.x * dz));
    const float wx = q2.y, wy = q2.z, wz = q2.w;
    PairGeom g;
    g.a = fmaf(px, px, fmaf(py, py, pz * pz));
    g.pw = fmaf(px, wx, fmaf(py, wy, pz * wz));
    const float cx = fmaf(wy, pz, -wz * py);
    const float cy = fmaf(wz, px, -wx * pz);
    const float cz = fmaf(wx, py, -wy * px);
    g.c2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
    return g;
}

// The ray cuts the culling ellipsoid (m^2 <= k^2) at t > 0 (s* > 0, unless
// the light is inside the culling sphere).
__device__ __forceinline__ bool pair_hit(const PairGeom &g, float k2, bool inside) {
    return g.c2 <= k2 * g.a && (inside || g.pw > 0.0f);
}

// ---------------------------------------------------------------------------
// Build tile kernel (Eqs. 2-4 over one tile's Gaussian list).
//
// Candidates.  Inside one face of the atlas map the texel rays of a tile are
// an affine family d(x, y) = d_c + x E_x + y E_y of the tile-local texel
// offsets (x, y) from the tile centre: Eq. 6 is affine in (u, v) on each face
// of the octahedron, and a cube face is a central projection.  The culling
// test of a pair, |w' x M d|^2 <= k^2 |M d|^2, is homogeneous of degree 2 in
// d, so over a tile it is a conic Q(x, y) <= 0 whose six coefficients are
// formed once per (Gaussian, tile), with k^2 widened by CONIC_WIDEN.  Each
// tile row meets the conic in an interval of texels (two roots of a
// quadratic): the candidate mask.  Where the expansion about the tile centre
// could lose the margin to rounding (a Gaussian far smaller than the tile),
// where the tile spans two faces, or where the light is inside the culling
// sphere, every texel is a candidate.
//
// Evaluation.  The candidates of a staged chunk go to one list, record by
// record (each thread writes its record's candidates at an offset from a
// warp scan); warps take 32 consecutive candidates at a time.  A lane tests
// its candidate exactly (the test above in the Gaussian's whitened frame, as
// the culling defines it) and evaluates Eq. 3 at the shells on the chord of
// the hit through the culling ellipsoid.  Consecutive candidates are
// neighbouring texels of one Gaussian, whose chords cover about as many
// shells, so the lanes of a warp take their shell loops nearly in step.
// Increments accumulate per tile in shared memory; the last work item of a
// tile takes the shell prefix sum and T = exp(-tau) (Eq. 4).
// ---------------------------------------------------------------------------
constexpr int SHELL_TB0 = 107 << 23;       // float bits of 2^-20
constexpr int SHELL_NB = 512;              // 16 buckets per octave over [2^-20, 2^12) metres
constexpr float CONIC_WIDEN = 1.0f / 32.0f;
constexpr float CONIC_COND = 1.0f / 8192.0f;

// Records per warp group: two lanes per record (the tile's top and bottom
// halves).
constexpr int TG = 16;
constexpr int BT_WARPS = BT_THREADS / 32;

size_t build_smem_bytes(int K, int tile, int chunk) {
    (void)chunk;  // the work items' size only
    const int nt = tile * tile;
    return (size_t)BT_WARPS * 2 * TG * REC_F4 * sizeof(float4) +  // per warp: two staged record groups
           (size_t)nt * sizeof(float4) +                           // texel directions
           (size_t)(K + 1) * nt * sizeof(float) +                  // per-shell increments (+ a row past the last)
           (size_t)((K + 5) & ~3) * sizeof(float) +                // radii, a +inf sentinel and one more
           (size_t)BT_WARPS * TG * nt * sizeof(uint16_t) +         // per warp: the group's candidate list
           (size_t)SHELL_NB * sizeof(uint16_t) +                   // shell table
           (size_t)SHELL_NB * sizeof(float2) +                     // its first two radii
           (size_t)BT_WARPS * 2 * TG;                              // per warp: half-tile masks
}

// Candidate texels of one staged record in rows [h T/2, (h+1) T/2) of a T x T
// tile: out[i] = jl | (je << 8), the columns [jl, je) of row h T/2 + i (je <=
// jl: none).  The binning's half-tile bit h (1: rows [0, T/2), 2: rows
// [T/2, T)) must be set; face: (d_c, ok), E_x, E_y of the tile; rows_valid x
// cols_valid: texels inside the atlas.
template <int T>
__device__ __forceinline__ void cand_mask(const float4 &q0, const float4 &q1, const float4 &q2,
                                          const float4 &q3, int h, const float4 &fc,
                                          const float4 &fx, const float4 &fy, int rows_valid,
                                          int cols_valid, uint32_t (&out)[T / 2]) {
    constexpr float HC = 0.5f * (float)(T - 1);
    const bool inside = (__float_as_int(q3.z) >> 20) & 1;
    bool conic = fc.w != 0.0f && !inside;
    float q00 = 0.f, qx = 0.f, qy = 0.f, qxx = 0.f, qxy = 0.f, qyy = 0.f;
    if (conic) {
        const float wx = q2.y, wy = q2.z, wz = q2.w;
        auto mvec = [&](float x, float y, float z, float &a, float &b, float &c) {
            a = fmaf(q0.x, x, fmaf(q0.y, y, q0.z * z));
            b = fmaf(q0.w, x, fmaf(q1.x, y, q1.y * z));
            c = fmaf(q1.z, x, fmaf(q1.w, y, q2.x * z));
        };
        float p0x, p0y, p0z, pxx, pxy, pxz, pyx, pyy, pyz;
        mvec(fc.x, fc.y, fc.z, p0x, p0y, p0z);
        mvec(fx.x, fx.y, fx.z, pxx, pxy, pxz);
        mvec(fy.x, fy.y, fy.z, pyx, pyy, pyz);
        // c = w' x p
        const float c0x = fmaf(wy, p0z, -wz * p0y), c0y = fmaf(wz, p0x, -wx * p0z), c0z = fmaf(wx, p0y, -wy * p0x);
        const float cxx = fmaf(wy, pxz, -wz * pxy), cxy = fmaf(wz, pxx, -wx * pxz), cxz = fmaf(wx, pxy, -wy * pxx);
        const float cyx = fmaf(wy, pyz, -wz * pyy), cyy = fmaf(wz, pyx, -wx * pyz), cyz = fmaf(wx, pyy, -wy * pyx);
        auto dot = [](float ax, float ay, float az, float bx, float by, float bz) {
            return fmaf(ax, bx, fmaf(ay, by, az * bz));
        };
        const float P00 = dot(p0x, p0y, p0z, p0x, p0y, p0z), Pxx = dot(pxx, pxy, pxz, pxx, pxy, pxz),
                    Pyy = dot(pyx, pyy, pyz, pyx, pyy, pyz);
        const float P0x = dot(p0x, p0y, p0z, pxx, pxy, pxz), P0y = dot(p0x, p0y, p0z, pyx, pyy, pyz),
                    Pxy = dot(pxx, pxy, pxz, pyx, pyy, pyz);
        const float C00 = dot(c0x, c0y, c0z, c0x, c0y, c0z), Cxx = dot(cxx, cxy, cxz, cxx, cxy, cxz),
                    Cyy = dot(cyx, cyy, cyz, cyx, cyy, cyz);
        const float C0x = dot(c0x, c0y, c0z, cxx, cxy, cxz), C0y = dot(c0x, c0y, c0z, cyx, cyy, cyz),
                    Cxy = dot(cxx, cxy, cxz, cyx, cyy, cyz);
        const float K2 = q3.y * (1.0f + CONIC_WIDEN);
        q00 = fmaf(-K2, P00, C00);
        qx = 2.0f * fmaf(-K2, P0x, C0x);
        qy = 2.0f * fmaf(-K2, P0y, C0y);
        qxx = fmaf(-K2, Pxx, Cxx);
        qxy = 2.0f * fmaf(-K2, Pxy, Cxy);
        qyy = fmaf(-K2, Pyy, Cyy);
        // The expansion keeps its margin when the terms it sums are not far
        // larger than k^2 |M d|^2 over the tile (|M d| >= |p0|/2 there).
        const float h2 = HC * HC;
        const float B = 3.0f * (fmaf(h2, Cxx + Cyy, C00) + K2 * fmaf(h2, Pxx + Pyy, P00));
        conic = 2.0f * h2 * (Pxx + Pyy) <= 0.25f * P00 && B * CONIC_COND <= q3.y * P00;
    }
    float i2a = 0.0f;
    if (conic && qxx > 0.0f) i2a = __fdividef(0.5f, qxx);
#pragma unroll
    for (int rr = 0; rr < T / 2; ++rr) {
        const int i = h * (T / 2) + rr;
        int jl = 0, je = cols_valid;
        if (i >= rows_valid) {
            je = 0;
        } else if (conic && qxx > 0.0f) {
            const float y = (float)i - HC;
            const float Bc = fmaf(qxy, y, qx), C = fmaf(y, fmaf(qyy, y, qy), q00);
            const float disc = fmaf(-4.0f * qxx, C, Bc * Bc);
            if (disc < 0.0f) {
                je = 0;
            } else {
                const float sd = disc * rsqrt_approx(fmaxf(disc, 1e-37f));
                const float xl = fmaxf(fmaf(-Bc - sd, i2a, HC - 1e-3f), -1.0f);
                const float xr = fminf(fmaf(sd - Bc, i2a, HC + 1e-3f), (float)T);
                jl = max(__float2int_ru(xl), 0);
                je = min(__float2int_rd(xr) + 1, cols_valid);
            }
        }
        out[rr] = (uint32_t)jl | ((uint32_t)max(je, 0) << 8);
    }
}

// Persistent: blocks pull work items (a tile's list, or a piece of it) from
// an atomic counter.  8 warps; staged chunks of records double buffered.
// The tile kernel's work as a device function of a whole block (the build's
// own kernel, and the persistent frame kernel, call it): pulls work items
// until none are left.  smem4: the block's dynamic shared memory,
// build_smem_bytes(K, T, chunk) bytes.
template <typename OutT, int T>
__device__ __forceinline__ void tiles_worker(
    const float4 *__restrict__ brec, const uint32_t *__restrict__ vals,
    const Item *__restrict__ items, const unsigned long long *__restrict__ n_items_total,
    unsigned int *__restrict__ item_counter, const float *__restrict__ radii, int K, int H, int W,
    int tx, int n_tiles, int64_t N, int chunk, float *__restrict__ accum,
    unsigned int *__restrict__ done, OutT *__restrict__ atlas,
    unsigned long long *__restrict__ stats, const uint8_t *__restrict__ roi_mask,
    const int *__restrict__ roi_k, int map, float4 *smem4) {
    // roi_mask, roi_k (or nullptr): texels [L][H][W] and shell range [kmin,
    // kmax] per light of a region of interest; T = 1 outside it
    constexpr int NT = T * T;
    (void)chunk;
    float4 *stage = smem4;                                    // [BT_WARPS][2][TG * REC_F4]
    float4 *tdir = stage + BT_WARPS * 2 * TG * REC_F4;        // [NT] (dir, valid)
    float *D = reinterpret_cast<float *>(tdir + NT);          // [K + 1][NT]: row K takes mass past the last shell
    float *rs = D + (K + 1) * NT;                             // [K + 1]: the radii, then +inf
    uint16_t *cand = reinterpret_cast<uint16_t *>(rs + ((K + 5) & ~3));  // [BT_WARPS][TG * NT]
    uint16_t *stab = cand + BT_WARPS * TG * NT;               // [SHELL_NB]
    float2 *stabr = reinterpret_cast<float2 *>(stab + SHELL_NB);    // [SHELL_NB] (r_c, r_c+1), c = stab[b]
    uint8_t *smask = reinterpret_cast<uint8_t *>(stabr + SHELL_NB);  // [BT_WARPS][2][TG]
    __shared__ uint4 s_item;
    __shared__ int s_last;
    __shared__ float4 s_face[3];
    __shared__ unsigned long long s_cnt[3];

    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t HW = (int64_t)H * W;
    const unsigned long long total_items = *n_items_total;
    for (int k = tid; k < K; k += BT_THREADS) rs[k] = radii[k];
    if (tid == 0) rs[K] = rs[K + 1] = __int_as_float(0x7f800000);  // no shell past the last
    if (tid < 3) s_cnt[tid] = 0ull;
    __syncthreads();
    // stab[b] = #{k : r_k < t_b}, t_b the float with bits SHELL_TB0 + (b << 19)
    for (int b = tid; b < SHELL_NB; b += BT_THREADS) {
        const float tb = __int_as_float(SHELL_TB0 + (b << 19));
        int c = 0;
        while (c < K && rs[c] < tb) ++c;
        stab[b] = (uint16_t)c;
        stabr[b] = make_float2(rs[c], rs[c + 1]);
    }
    // a bucket holds several radii (radii closer than 1/16 octave, or outside
    // the table's range): the shell search then counts the radii one by one
    int several = 0;
    for (int k = tid; k + 1 < K; k += BT_THREADS) {
        const int bk = __float_as_int(rs[k]), bn = __float_as_int(rs[k + 1]);
        const bool out = bk <= SHELL_TB0 || bn - SHELL_TB0 >= (SHELL_NB << 19);
        several |= out || ((bk - SHELL_TB0) >> 19) == ((bn - SHELL_TB0) >> 19);
    }
    const bool step_more = __syncthreads_or(several) != 0;
    unsigned int n_cand = 0, n_hit = 0, n_shell = 0;
    for (;;) {
        if (tid == 0) {
            const unsigned it = atomicAdd(item_counter, 1u);
            s_item = it < total_items ? *reinterpret_cast<const uint4 *>(items + it)
                                      : make_uint4(0xffffffffu, 0u, 0u, 0u);
        }
        __syncthreads();
        const uint4 item = s_item;
        if (item.x == 0xffffffffu) break;
        const uint32_t key = item.x, start = item.y, end = item.z, n_items = item.w;
        const int l = key / n_tiles, t = key - l * n_tiles;
        const int tile_i = t / tx, tile_j = t - tile_i * tx;
        const int i0 = tile_i * T, j0 = tile_j * T;
        const int rows_valid = min(T, H - i0), cols_valid = min(T, W - j0);
        for (int e = tid; e < (K + 1) * NT; e += BT_THREADS) D[e] = 0.0f;
        for (int e = tid; e < NT; e += BT_THREADS) {
            const int i = i0 + e / T, j = j0 + e % T;
            float x, y, z;
            if (map == MAP_CUBE) {
                const int f = min(i / W, 5);
                const float u = (2.0f * j + 1.0f) / W - 1.0f, v = (2.0f * (i - f * W) + 1.0f) / W - 1.0f;
                int aF, aU, aV;
                float sF, sU, sV;
                cube_axes(f, aF, aU, aV, sF, sU, sV);
                x = aF == 0 ? sF : aU == 0 ? sU * u : sV * v;
                y = aF == 1 ? sF : aU == 1 ? sU * u : sV * v;
                z = aF == 2 ? sF : aU == 2 ? sU * u : sV * v;
            } else {
                const float u = (2.0f * j + 1.0f) / W - 1.0f, v = (2.0f * i + 1.0f) / H - 1.0f;
                z = 1.0f - fabsf(u) - fabsf(v), x = u, y = v;
                if (z < 0.0f) {
                    x = (u >= 0.f ? 1.f : -1.f) * (1.0f - fabsf(v));
                    y = (v >= 0.f ? 1.f : -1.f) * (1.0f - fabsf(u));
                }
            }
            const float inv = rsqrtf(x * x + y * y + z * z);
            tdir[e] = make_float4(x * inv, y * inv, z * inv, (i < H && j < W) ? 1.0f : 0.0f);
        }
        if (tid == 0) {
            // the tile's affine ray family d_c + x E_x + y E_y (texel offsets x, y)
            float dc0, dc1, dc2, ex0 = 0.f, ex1 = 0.f, ex2 = 0.f, ey0 = 0.f, ey1 = 0.f, ey2 = 0.f;
            bool ok = true;
            if (map == MAP_CUBE) {
                const int f = min(i0 / W, 5);
                int aF, aU, aV;
                float sF, sU, sV;
                cube_axes(f, aF, aU, aV, sF, sU, sV);
                const float du = 2.0f / W;
                const float uc = (float)(2 * j0 + T) / W - 1.0f, vc = (float)(2 * (i0 - f * W) + T) / W - 1.0f;
                dc0 = aF == 0 ? sF : aU == 0 ? sU * uc : sV * vc;
                dc1 = aF == 1 ? sF : aU == 1 ? sU * uc : sV * vc;
                dc2 = aF == 2 ? sF : aU == 2 ? sU * uc : sV * vc;
                ex0 = aU == 0 ? sU * du : 0.f;
                ex1 = aU == 1 ? sU * du : 0.f;
                ex2 = aU == 2 ? sU * du : 0.f;
                ey0 = aV == 0 ? sV * du : 0.f;
                ey1 = aV == 1 ? sV * du : 0.f;
                ey2 = aV == 2 ? sV * du : 0.f;
            } else {
                const float du = 2.0f / W, dv = 2.0f / H;
                const float uc = (float)(2 * j0 + T) / W - 1.0f, vc = (float)(2 * i0 + T) / H - 1.0f;
                const float ua = (2.0f * j0 + 1.0f) / W - 1.0f, ub = (2.0f * (j0 + cols_valid - 1) + 1.0f) / W - 1.0f;
                const float va = (2.0f * i0 + 1.0f) / H - 1.0f, vb = (2.0f * (i0 + rows_valid - 1) + 1.0f) / H - 1.0f;
                const float su = ua >= 0.f ? 1.f : -1.f, sv = va >= 0.f ? 1.f : -1.f;
                ok = (ub >= 0.f) == (ua >= 0.f) && (vb >= 0.f) == (va >= 0.f);
                const float s00 = fabsf(ua) + fabsf(va), s01 = fabsf(ub) + fabsf(va);
                const float s10 = fabsf(ua) + fabsf(vb), s11 = fabsf(ub) + fabsf(vb);
                const bool inner = fmaxf(fmaxf(s00, s01), fmaxf(s10, s11)) <= 1.0f;
                const bool outer = fminf(fminf(s00, s01), fminf(s10, s11)) >= 1.0f;
                ok = ok && (inner || outer);
                // inner face: d = (u, v, 1 - su u - sv v); outer (folded) face:
                // d = (su (1 - sv v), sv (1 - su u), 1 - su u - sv v)
                dc2 = 1.0f - su * uc - sv * vc;
                ex2 = -su * du;
                ey2 = -sv * dv;
                if (inner) {
                    dc0 = uc;
                    dc1 = vc;
                    ex0 = du;
                    ey1 = dv;
                } else {
                    dc0 = su - su * sv * vc;
                    dc1 = sv - su * sv * uc;
                    ex1 = -su * sv * du;
                    ey0 = -su * sv * dv;
                }
            }
            s_face[0] = make_float4(dc0, dc1, dc2, ok ? 1.f : 0.f);
            s_face[1] = make_float4(ex0, ex1, ex2, 0.f);
            s_face[2] = make_float4(ey0, ey1, ey2, 0.f);
        }
        const float4 *src = brec + (int64_t)l * N * REC_F4;
        const int nrec = (int)(end - start);
        const int ngroups = (nrec + TG - 1) / TG;
        // Warp w takes the record groups w, w + BT_WARPS, ... of the item (TG
        // consecutive records each), staged in its own slice of shared memory
        // one group ahead; it forms their candidate list in its own slice and
        // evaluates it, with no block barrier until the item's end.  Staging:
        // lane l copies the float4 parts e = l, l + 32 of the group (record
        // e / REC_F4, part e % REC_F4).
        const int warp = tid >> 5;
        float4 *wst = stage + warp * 2 * TG * REC_F4;
        uint8_t *wsm = smask + warp * 2 * TG;
        uint16_t *wc = cand + warp * TG * NT;
        auto load_idx = [&](int g, uint32_t (&gi)[2]) {
            const int base = (int)start + g * TG, cnt = min(TG, (int)end - base);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int e = lane + 32 * hh;
                gi[hh] = e < cnt * REC_F4 ? __ldg(vals + base + e / REC_F4) : 0u;
            }
        };
        auto issue = [&](int g, int buf, const uint32_t (&gi)[2]) {
            const int base = (int)start + g * TG, cnt = min(TG, (int)end - base);
            float4 *dst = wst + buf * TG * REC_F4;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int e = lane + 32 * hh;
                if (e < cnt * REC_F4) {
                    cp_async16(dst + e, src + (int64_t)(gi[hh] & VAL_IDX) * REC_F4 + e % REC_F4);
                    if (e % REC_F4 == 0) wsm[buf * TG + e / REC_F4] = (uint8_t)(gi[hh] >> 30);
                }
            }
            cp_async_commit();
        };
        uint32_t gnext[2] = {0u, 0u};
        if (warp < ngroups) {
            uint32_t g0[2];
            load_idx(warp, g0);
            issue(warp, 0, g0);
            if (warp + BT_WARPS < ngroups) load_idx(warp + BT_WARPS, gnext);
        }
        __syncthreads();  // D, the texel directions and the tile's ray family are set
        for (int g = warp, it = 0; g < ngroups; g += BT_WARPS, ++it) {
            const int buf = it & 1;
            if (g + BT_WARPS < ngroups) {
                // the other buffer's group was consumed before the previous __syncwarp
                issue(g + BT_WARPS, buf ^ 1, gnext);
                if (g + 2 * BT_WARPS < ngroups) load_idx(g + 2 * BT_WARPS, gnext);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();  // every lane's copies of this group are in shared memory
            const float4 *st = wst + buf * TG * REC_F4;
            const int cnt = min(TG, (int)end - ((int)start + g * TG));
            // candidate list: lanes 2r and 2r + 1 write the candidates of record r
            // in the top and bottom half of the tile at offsets from a warp scan
            int total;
            {
                uint32_t iv[T / 2];
#pragma unroll
                for (int rr = 0; rr < T / 2; ++rr) iv[rr] = 0u;
                const int r = lane >> 1, h = lane & 1;
                int nr = 0;
                if (r < cnt && ((wsm[buf * TG + r] >> h) & 1u)) {
                    cand_mask<T>(st[r * REC_F4], st[r * REC_F4 + 1], st[r * REC_F4 + 2], st[r * REC_F4 + 3],
                                 h, s_face[0], s_face[1], s_face[2], rows_valid, cols_valid, iv);
#pragma unroll
                    for (int rr = 0; rr < T / 2; ++rr) nr += max((int)(iv[rr] >> 8) - (int)(iv[rr] & 255u), 0);
                }
                int incl = nr;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULLMASK, incl, o);
                    if (lane >= o) incl += v;
                }
                total = __shfl_sync(FULLMASK, incl, 31);
                int pos = incl - nr;
#pragma unroll
                for (int rr = 0; rr < T / 2; ++rr) {
                    const int id0 = (r << 8) | ((h * (T / 2) + rr) * T);
                    for (int j = (int)(iv[rr] & 255u); j < (int)(iv[rr] >> 8); ++j) wc[pos++] = (uint16_t)(id0 + j);
                }
            }
            __syncwarp();
            if (lane == 0) n_cand += (unsigned)total;
            // batches of 32 consecutive candidates; the body is straight-line code
            // with predicated deposits (lanes past the list's end or without a hit
            // deposit nothing)
            // each batch's candidate ids are read one batch ahead
            uint32_t id_next = lane < total ? wc[lane] : 0u;
            for (int f0 = 0; f0 < total; f0 += 32) {
                const bool valid = f0 + lane < total;
                const uint32_t id = id_next;
                id_next = f0 + 32 + lane < total ? wc[f0 + 32 + lane] : 0u;
                const int r = (int)(id >> 8), tex = (int)(id & 255u);
                const float4 q0 = st[r * REC_F4], q1 = st[r * REC_F4 + 1], q2 = st[r * REC_F4 + 2],
                             q3 = st[r * REC_F4 + 3];
                const float4 dd = tdir[tex];
                const PairGeom g = pair_geom(q0, q1, q2, dd.x, dd.y, dd.z);
                const bool inside = (__float_as_int(q3.z) >> 20) & 1;
                const bool hit = valid && pair_hit(g, q3.y, inside);
                n_hit += hit ? 1u : 0u;
                const float rsa = rsqrt_approx(g.a);
                const float ia = rsa * rsa;
                const float m2 = g.c2 * ia;   // c - b^2/a
                const float ss = g.pw * ia;   // closest approach s* = -b/a
                // the chord through the culling ellipsoid, s* +- sqrt((k^2 - m^2)/a):
                // the ray's mass outside it is at most eps_cull, so shells before it
                // get nothing and the first shell past it the whole remaining mass
                const float c2h = fmaxf(q3.y - m2, 1e-30f);
                const float half = c2h * rsqrt_approx(c2h) * rsa;
                const float lo = ss - half, hi = ss + half;
                // first shell at or past the chord's start: the table's bucket holds
                // at most one radius (else step_more is set and the radii are counted)
                // (the bucket's first two radii come from a table beside it, read
                // together with it; rk = r_k is carried into the shell loop)
                int k;
                float rk;
                if (!step_more) {
                    const int bk = max(min((__float_as_int(lo) - SHELL_TB0) >> 19, SHELL_NB - 1), 0);
                    k = stab[bk];
                    const float2 rab = stabr[bk];
                    const float ra = rab.x, rb = rab.y;
                    rk = ra < lo ? rb : ra;
                    k += ra < lo ? 1 : 0;
                } else {
                    k = 0;
                    while (k < K && rs[k] < lo) ++k;
                    rk = rs[k];
                }
                const float A0 = q3.x * rsa;                  // beta sqrt(pi/(2a))
                const float hh = g.a * rsa * 0.70710678118f;  // sqrt(a/2)
                const float hm2 = -0.72134752044f * m2;       // -m^2/2 log2(e)
                const float full = 2.0f * A0 * ex2_approx(hm2);
                const float hs = hh * ss;
                float F0 = 0.0f;
                if (__any_sync(FULLMASK, inside)) F0 = inside ? mass_below(-hs, A0, hm2, full) : 0.0f;
                const int k0 = k;
                float Gprev = 0.0f;
                // shells on the chord (most hits have none or one); rk = r_k is
                // carried in a register (the deposits may alias the radii for
                // the compiler, which would otherwise load it twice a pass)
                bool more = hit && rk <= hi;
                while (__any_sync(FULLMASK, more)) {
                    const float G = mass_below(fmaf(hh, rk, -hs), A0, hm2, full) - F0;
                    if (more) {
                        atomicAdd(D + k * NT + tex, fmaxf(G - Gprev, 0.0f));
                        Gprev = fmaxf(G, Gprev);
                        ++k;
                        rk = rs[k];
                    }
                    more = more && rk <= hi;
                }
                n_shell += (unsigned)(k - k0);
                if (hit) atomicAdd(D + k * NT + tex, fmaxf(full - F0 - Gprev, 0.0f));  // row K: unused
            }
            __syncwarp();  // the group's records and list are no longer read
        }
        __syncthreads();
        // ---- finalize: prefix over shells, T = exp(-tau) (Eq. 4) ----
        const int kmin = roi_k ? roi_k[2 * l] : 0, kmax = roi_k ? roi_k[2 * l + 1] : K - 1;
        if (n_items == 1) {
            for (int e = tid; e < NT; e += BT_THREADS) {
                if (tdir[e].w == 0.0f) continue;
                const int i = i0 + e / T, j = j0 + e % T;
                OutT *dst = atlas + (int64_t)l * K * HW + (int64_t)i * W + j;
                const bool in = !roi_mask || roi_mask[(int64_t)l * HW + (int64_t)i * W + j];
                float tau = 0.0f, Tprev = 1.0f;
                for (int k = 0; k < K; ++k) {
                    tau += D[k * NT + e];
                    const float Tk = fminf(expf(-tau), Tprev);  // kept non-increasing in k
                    Tprev = Tk;
                    dst[k * HW] = to_store<OutT>(in && k >= kmin && k <= kmax ? Tk : 1.0f);
                }
            }
        } else {
            for (int e = tid; e < K * NT; e += BT_THREADS) {
                const int k = e / NT, te = e - k * NT;
                const float v = D[e];
                if (v == 0.0f || tdir[te].w == 0.0f) continue;
                const int i = i0 + te / T, j = j0 + te % T;
                atomicAdd(accum + ((int64_t)l * K + k) * HW + (int64_t)i * W + j, v);
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(done + key, 1u) == n_items - 1u;
            __syncthreads();
            if (s_last) {
                __threadfence();
                for (int e = tid; e < NT; e += BT_THREADS) {
                    if (tdir[e].w == 0.0f) continue;
                    const int i = i0 + e / T, j = j0 + e % T;
                    OutT *dst = atlas + (int64_t)l * K * HW + (int64_t)i * W + j;
                    float *acc = accum + (int64_t)l * K * HW + (int64_t)i * W + j;
                    const bool in = !roi_mask || roi_mask[(int64_t)l * HW + (int64_t)i * W + j];
                    float tau = 0.0f, Tprev = 1.0f;
                    for (int k = 0; k < K; ++k) {
                        tau += __ldcg(acc + k * HW);
                        acc[k * HW] = 0.0f;  // ready for the next build
                        const float Tk = fminf(expf(-tau), Tprev);
                        Tprev = Tk;
                        dst[k * HW] = to_store<OutT>(in && k >= kmin && k <= kmax ? Tk : 1.0f);
                    }
                }
                if (tid == 0) done[key] = 0u;
            }
        }
        __syncthreads();  // shared state is reused by the next item
    }
    if (stats) {
        if (n_cand) atomicAdd(&s_cnt[0], (unsigned long long)n_cand);
        if (n_hit) atomicAdd(&s_cnt[1], (unsigned long long)n_hit);
        if (n_shell) atomicAdd(&s_cnt[2], (unsigned long long)n_shell);
        __syncthreads();
        if (tid < 3) atomicAdd(stats + tid, s_cnt[tid]);
    }
}

}  // namespace
}  // namespace dgsm
