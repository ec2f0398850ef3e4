// render.cu -- 3DGS splatting on sm_103a for the cubemap probe of Sec. 3.4
// (the scene on the six 90-degree faces at the avatar; the SH fit of Eq. 7
// takes the faces' texels as its samples) and for the final composite of the
// relit avatar in the shadowed scene, seen by pinhole cameras.
//
// Pipeline per call (all on the caller's stream), for n_views cameras:
//   splat_prep_kernel   per Gaussian and view (a splat): view coordinates,
//                       the EWA screen covariance (Jacobian of the pinhole
//                       projection at the mean), its inverse, its payload,
//                       its depth and a conservative rectangle of 8x8 tiles
//                       around the 3-sigma ellipse
//   scan, compaction    the splats that reach a tile
//   radix sort          those splats by depth (stable: ties by Gaussian index)
//   scan                pair offsets of the splats in depth order (one host
//                       sync for the pair count)
//   splat_pairs_kernel  the (tile, splat) pairs in depth order, every block
//                       spreading its splats' pairs over all of its threads
//   radix sort          the pairs stably by tile: each tile's splats front
//                       to back
//   splat_ranges_kernel [start, end) of every tile
//   segment kernels     every tile's list cut into segments of `seg` splats,
//                       seg sized so that the segments fill the GPU
//   splat_segment_kernel one block per segment, one thread per pixel: the
//                       segment's splats composited front to back,
//                       C += alpha T c, T *= 1 - alpha (local T)
//   splat_merge_kernel  per pixel, the segments in order:
//                       C = C_0 + T_0 (C_1 + T_1 (C_2 + ...))
// Every splat within 3 sigma of a pixel is composited; a segment, and the
// merge, stop once their transmittance is below T_CUT, which changes the
// colour by less than T_CUT times the brightest splat colour.
// The pixel-inclusion decision (Mahalanobis distance <= 3) and the depth
// order use IEEE single-precision operations in a fixed order, so they are
// reproducible on the CPU; the tiles only accelerate it.
#include <algorithm>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int RT = 8;                // render tile edge, pixels
constexpr int RT_PIX = RT * RT;      // threads per render block
constexpr float LOWPASS = 0.3f;      // screen-space dilation, pixel^2
constexpr float JAC_LIMIT = 1.3f;    // Jacobian evaluated within 1.3 x the half field of view
constexpr float T_CUT = 1e-6f;       // transmittance below which the rest is left out
constexpr int SEG_MIN = 256;         // least splats per segment of a tile's list
constexpr float ALPHA_MAX = 0.99f;
constexpr int CAM_F = 16;            // floats per camera: R (9, rows x, y, forward), position (3), fx, fy, cx, cy

// Face f of the cube: forward axis F and the axes U, V along which the face's
// texel coordinates u (columns) and v (rows) grow, as signed unit axes
// (axis index, sign).  Direction of texel (u, v) = F + u U + v V.
__constant__ int c_face_axis[6][3] = {{0, 2, 1}, {0, 2, 1}, {1, 0, 2}, {1, 0, 2}, {2, 0, 1}, {2, 0, 1}};
__constant__ float c_face_sign[6][3] = {{1, -1, -1}, {-1, 1, -1}, {1, 1, 1}, {-1, 1, -1}, {1, 1, -1},
                                        {-1, -1, -1}};

struct Splat {
    float mx, my;      // mean in the image, pixels (pixel j's centre at j + 0.5)
    float A, B, C;     // inverse screen covariance [[A, B], [B, C]]
    float tz;          // depth along the camera's forward axis
    int rx, ry;        // half-widths of the pixel box around the mean
    bool ok;
};

// The Gaussian's splat in camera c (cam: 16 floats) for a W x H image.  All
// steps are IEEE single operations in this order (the CPU oracle repeats
// them): t = mu - position; (tx, ty, tz) = R t (rows x, y, forward);
// u = tx / tz, v = ty / tz; mean = (fx u + cx, fy v + cy); G = R (R_g diag(s))
// column by column; p1 = g_x - u' g_z, p2 = g_y - v' g_z with u', v' clamped
// to 1.3 x the half field of view; hx = fx / tz, hy = fy / tz; the screen
// covariance [[hx^2 p1.p1, hx hy p1.p2], [., hy^2 p2.p2]] + LOWPASS I and
// its inverse.
__device__ __forceinline__ Splat make_splat(const float *mu, const float *Rs, const float *cam, int W, int H,
                                            float near) {
    Splat sp;
    sp.ok = false;
    const float *R = cam;
    const float t0 = xsub(mu[0], cam[9]), t1 = xsub(mu[1], cam[10]), t2 = xsub(mu[2], cam[11]);
    const float tx = xdot(R[0], R[1], R[2], t0, t1, t2);
    const float ty = xdot(R[3], R[4], R[5], t0, t1, t2);
    const float tz = xdot(R[6], R[7], R[8], t0, t1, t2);
    sp.tz = tz;
    if (!(tz > near)) return sp;
    const float fx = cam[12], fy = cam[13];
    const float u = xdiv(tx, tz), v = xdiv(ty, tz);
    sp.mx = xadd(xmul(fx, u), cam[14]);
    sp.my = xadd(xmul(fy, v), cam[15]);
    float gx[3], gy[3], gz[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gx[k] = xdot(R[0], R[1], R[2], Rs[k], Rs[3 + k], Rs[6 + k]);
        gy[k] = xdot(R[3], R[4], R[5], Rs[k], Rs[3 + k], Rs[6 + k]);
        gz[k] = xdot(R[6], R[7], R[8], Rs[k], Rs[3 + k], Rs[6 + k]);
    }
    const float limx = xmul(JAC_LIMIT, xdiv(xmul(0.5f, (float)W), fx));
    const float limy = xmul(JAC_LIMIT, xdiv(xmul(0.5f, (float)H), fy));
    const float uc = fminf(fmaxf(u, -limx), limx), vc = fminf(fmaxf(v, -limy), limy);
    float p1[3], p2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p1[k] = xsub(gx[k], xmul(uc, gz[k]));
        p2[k] = xsub(gy[k], xmul(vc, gz[k]));
    }
    const float n11 = xdot(p1[0], p1[1], p1[2], p1[0], p1[1], p1[2]);
    const float n12 = xdot(p1[0], p1[1], p1[2], p2[0], p2[1], p2[2]);
    const float n22 = xdot(p2[0], p2[1], p2[2], p2[0], p2[1], p2[2]);
    const float hx = xdiv(fx, tz), hy = xdiv(fy, tz);
    const float a = xadd(xmul(xmul(hx, hx), n11), LOWPASS);
    const float b = xmul(xmul(hx, hy), n12);
    const float c = xadd(xmul(xmul(hy, hy), n22), LOWPASS);
    const float det = xsub(xmul(a, c), xmul(b, b));
    if (!(det > 0.0f)) return sp;
    sp.A = xdiv(c, det);
    sp.B = xdiv(-b, det);
    sp.C = xdiv(a, det);
    // the box that bounds the 3-sigma ellipse (half-widths 3 sqrt(a), 3 sqrt(c)),
    // with a pixel of margin: it only selects tiles, the ellipse test decides
    const float ex = 3.0f * sqrtf(a) * 1.001f + 1.0f, ey = 3.0f * sqrtf(c) * 1.001f + 1.0f;
    if (!(ex < 1e6f) || !(ey < 1e6f) || !(fabsf(sp.mx) < 1e7f) || !(fabsf(sp.my) < 1e7f)) return sp;
    sp.rx = (int)ceilf(ex);
    sp.ry = (int)ceilf(ey);
    sp.ok = true;
    return sp;
}

// Mahalanobis distance squared of pixel centre (px, py) from the splat, in a fixed order.
__device__ __forceinline__ float splat_m2(float px, float py, float mx, float my, float A, float B, float C) {
    const float dx = xsub(px, mx), dy = xsub(py, my);
    return xadd(xadd(xmul(A, xmul(dx, dx)), xmul(xmul(2.0f, B), xmul(dx, dy))), xmul(C, xmul(dy, dy)));
}

// R diag(s) of a Gaussian (quaternion w, x, y, z normalised first), row-major,
// in IEEE single operations in a fixed order (part of the inclusion decision).
__device__ __forceinline__ void rot_scale(const float *q, const float *s, float *Rs) {
    const float n = xsqrt(xadd(xadd(xadd(xmul(q[0], q[0]), xmul(q[1], q[1])), xmul(q[2], q[2])), xmul(q[3], q[3])));
    const float w = xdiv(q[0], n), x = xdiv(q[1], n), y = xdiv(q[2], n), z = xdiv(q[3], n);
    const float xx = xmul(x, x), yy = xmul(y, y), zz = xmul(z, z);
    const float xy = xmul(x, y), xz = xmul(x, z), yz = xmul(y, z);
    const float wx = xmul(w, x), wy = xmul(w, y), wz = xmul(w, z);
    const float R[9] = {xsub(1.0f, xmul(2.0f, xadd(yy, zz))), xmul(2.0f, xsub(xy, wz)), xmul(2.0f, xadd(xz, wy)),
                        xmul(2.0f, xadd(xy, wz)), xsub(1.0f, xmul(2.0f, xadd(xx, zz))), xmul(2.0f, xsub(yz, wx)),
                        xmul(2.0f, xsub(xz, wy)), xmul(2.0f, xadd(yz, wx)), xsub(1.0f, xmul(2.0f, xadd(xx, yy)))};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) Rs[3 * r + k] = xmul(R[3 * r + k], s[k]);
}

// Tile range of a splat in its image ([i0, i1) x [j0, j1)); empty if off the image.
__device__ __forceinline__ void splat_tiles(const Splat &sp, int ntx, int nty, int &i0, int &i1, int &j0,
                                            int &j1) {
    const float lo_x = sp.mx - (float)sp.rx, hi_x = sp.mx + (float)sp.rx;
    const float lo_y = sp.my - (float)sp.ry, hi_y = sp.my + (float)sp.ry;
    j0 = (int)fminf(fmaxf(floorf(lo_x / RT), 0.0f), (float)ntx);
    j1 = (int)fminf(fmaxf(floorf(hi_x / RT) + 1.0f, 0.0f), (float)ntx);
    i0 = (int)fminf(fmaxf(floorf(lo_y / RT), 0.0f), (float)nty);
    i1 = (int)fminf(fmaxf(floorf(hi_y / RT) + 1.0f, 0.0f), (float)nty);
    if (j1 < j0) j1 = j0;
    if (i1 < i0) i1 = i0;
}

// Splat sid = g n_views + v (Gaussian g, view v): payload (mx, my, A, B),
// (C, opacity, tz, g), (r, g, b, 0); depth key (the bits of tz > 0 order like
// its values); 1 if it reaches a tile; tile count; tile rectangle and view
// (i0 | j0 << 16, width in tiles | view << 16).
__global__ void __launch_bounds__(256) splat_prep_kernel(
    const float *__restrict__ means, const float *__restrict__ scales, const float *__restrict__ quats,
    const float *__restrict__ opac, const float *__restrict__ colors, int64_t n, const float *__restrict__ cams,
    int n_views, int W, int H, float near, uint32_t *__restrict__ dkey, uint32_t *__restrict__ live,
    uint32_t *__restrict__ counts, uint2 *__restrict__ rect, float4 *__restrict__ payload) {
    __shared__ float scam[64 * CAM_F];
    for (int k = threadIdx.x; k < n_views * CAM_F; k += blockDim.x) scam[k] = cams[k];
    __syncthreads();
    const int ntx = (W + RT - 1) / RT, nty = (H + RT - 1) / RT;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const float al = opac[g];
        float Rs[9];
        if (al > 0.0f) rot_scale(quats + 4 * g, scales + 3 * g, Rs);
        for (int v = 0; v < n_views; ++v) {
            const size_t sid = (size_t)g * n_views + v;
            uint32_t key = 0xffffffffu, c = 0u;
            uint2 rc = make_uint2(0u, 0u);
            if (al > 0.0f) {
                const Splat sp = make_splat(means + 3 * g, Rs, scam + CAM_F * v, W, H, near);
                if (sp.ok) {
                    int i0, i1, j0, j1;
                    splat_tiles(sp, ntx, nty, i0, i1, j0, j1);
                    if (i1 > i0 && j1 > j0) {
                        key = __float_as_uint(sp.tz);
                        c = (uint32_t)((i1 - i0) * (j1 - j0));
                        rc = make_uint2((uint32_t)i0 | ((uint32_t)j0 << 16), (uint32_t)(j1 - j0) | ((uint32_t)v << 16));
                        payload[3 * sid] = make_float4(sp.mx, sp.my, sp.A, sp.B);
                        payload[3 * sid + 1] = make_float4(sp.C, al, sp.tz, __int_as_float((int)g));
                        payload[3 * sid + 2] = make_float4(colors[3 * g], colors[3 * g + 1], colors[3 * g + 2], 0.0f);
                    }
                }
            }
            dkey[sid] = key;
            live[sid] = c > 0u ? 1u : 0u;
            counts[sid] = c;
            rect[sid] = rc;
        }
    }
}

// The splats that reach a tile, in index order (pos: exclusive scan of the
// flags): their depth keys and indices, for the depth sort.
__global__ void compact_splats_kernel(const uint32_t *__restrict__ dkey, const uint32_t *__restrict__ counts,
                                      const uint32_t *__restrict__ pos, int64_t ns, uint32_t *__restrict__ ckey,
                                      uint32_t *__restrict__ csid) {
    for (int64_t sid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sid < ns;
         sid += (int64_t)gridDim.x * blockDim.x) {
        if (counts[sid] == 0u) continue;
        const uint32_t k = pos[sid];
        ckey[k] = dkey[sid];
        csid[k] = (uint32_t)sid;
    }
}

// Tile counts of the splats in depth order (0 past the nv live splats).
__global__ void sorted_counts_kernel(const uint32_t *__restrict__ order, const uint32_t *__restrict__ counts,
                                     const unsigned long long *__restrict__ d_nv, int64_t ns,
                                     uint32_t *__restrict__ out) {
    const int64_t nv = (int64_t)*d_nv;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < ns; r += (int64_t)gridDim.x * blockDim.x)
        out[r] = r < nv ? counts[order[r]] : 0u;
}

// The pairs of the splats in depth order: a block takes PAIR_T consecutive
// splats and cuts their pairs into tiles of PAIR_T x PAIR_U.  In a tile each
// thread finds the splat of its first pair by a binary search of the splats'
// offsets in shared memory, then walks PAIR_U consecutive pairs over the
// splats' tile rectangles (row by row); the tile is staged in shared memory
// and stored coalesced.  A splat over thousands of tiles does not hold one
// thread.
constexpr int PAIR_T = 256;
constexpr int PAIR_U = 8;
__global__ void __launch_bounds__(PAIR_T) splat_pairs_kernel(
    const uint32_t *__restrict__ order, const uint32_t *__restrict__ off, const uint2 *__restrict__ rect,
    int64_t ns, const unsigned long long *__restrict__ d_nv, const unsigned long long *__restrict__ d_total,
    int ntx, int nty, uint32_t *__restrict__ tkey, uint32_t *__restrict__ pid) {
    __shared__ uint32_t s_off[PAIR_T + 1];
    __shared__ uint32_t s_sid[PAIR_T];
    __shared__ uint32_t s_key[PAIR_T * PAIR_U], s_pid[PAIR_T * PAIR_U];
    const uint32_t P = (uint32_t)*d_total;
    const int64_t nv = (int64_t)*d_nv;
    const int tid = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * PAIR_T; base < ns; base += (int64_t)gridDim.x * PAIR_T) {
        __syncthreads();  // the previous range is no longer read
        const int64_t r = base + tid;
        s_off[tid] = r < ns ? off[r] : P;
        s_sid[tid] = r < nv ? order[r] : 0u;
        if (tid == 0) s_off[PAIR_T] = base + PAIR_T < ns ? off[base + PAIR_T] : P;
        __syncthreads();
        const uint32_t p1 = s_off[PAIR_T];
        for (uint32_t t0 = s_off[0]; t0 < p1; t0 += PAIR_T * PAIR_U) {
            const uint32_t q0 = t0 + (uint32_t)tid * PAIR_U;
            if (q0 < p1) {
                // the last splat of the block whose offset is <= q0 (splats
                // without pairs share the offset of the next one, before it)
                int lo = 0, hi = PAIR_T - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= q0) lo = mid; else hi = mid - 1;
                }
                uint32_t sid = s_sid[lo], left = s_off[lo + 1] - q0;
                uint2 rc = rect[sid];
                uint32_t i0 = rc.x & 0xffffu, j0 = rc.x >> 16, w = rc.y & 0xffffu, v = rc.y >> 16;
                const uint32_t local = q0 - s_off[lo], di = local / w;
                uint32_t i = i0 + di, j = j0 + (local - di * w);
                const int nu = (int)min((uint32_t)PAIR_U, p1 - q0);
                for (int u = 0; u < nu; ++u) {
                    if (left == 0u) {  // the next splat with pairs
                        do {
                            ++lo;
                        } while (s_off[lo + 1] == s_off[lo]);
                        sid = s_sid[lo];
                        left = s_off[lo + 1] - s_off[lo];
                        rc = rect[sid];
                        i0 = rc.x & 0xffffu;
                        j0 = rc.x >> 16;
                        w = rc.y & 0xffffu;
                        v = rc.y >> 16;
                        i = i0;
                        j = j0;
                    }
                    s_key[tid * PAIR_U + u] = (v * (uint32_t)nty + i) * (uint32_t)ntx + j;
                    s_pid[tid * PAIR_U + u] = sid;
                    --left;
                    if (++j == j0 + w) {
                        j = j0;
                        ++i;
                    }
                }
            }
            __syncthreads();
            const uint32_t cnt = min((uint32_t)(PAIR_T * PAIR_U), p1 - t0);
            for (uint32_t x = (uint32_t)tid; x < cnt; x += PAIR_T) {
                tkey[t0 + x] = s_key[x];
                pid[t0 + x] = s_pid[x];
            }
            __syncthreads();
        }
    }
}

__global__ void splat_ranges_kernel(const uint32_t *__restrict__ keys, const unsigned long long *__restrict__ d_n,
                                    uint32_t *__restrict__ ts, uint32_t *__restrict__ te) {
    const unsigned long long n = *d_n;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ts[k] = (uint32_t)i;
        if (i + 1 == n || keys[i + 1] != k) te[k] = (uint32_t)(i + 1);
    }
}

// Segments: seg_cnt[t] = ceil(list length / seg), at least 1 (an empty tile
// still writes its pixels).
__global__ void seg_count_kernel(const uint32_t *__restrict__ ts, const uint32_t *__restrict__ te, int64_t n_tiles,
                                 uint32_t seg, uint32_t *__restrict__ seg_cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) seg_cnt[t] = max(1u, (te[t] - ts[t] + seg - 1) / seg);
}

// seg = (tile, start, end, index of the tile's first segment)
__global__ void seg_fill_kernel(const uint32_t *__restrict__ ts, const uint32_t *__restrict__ te, int64_t n_tiles,
                                uint32_t seg, const uint32_t *__restrict__ seg_off, uint4 *__restrict__ segs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t s0 = ts[t], e0 = te[t], o = seg_off[t];
    const uint32_t n = max(1u, (e0 - s0 + seg - 1) / seg);
    for (uint32_t k = 0; k < n; ++k)
        segs[o + k] = make_uint4((uint32_t)t, s0 + k * seg, min(s0 + (k + 1) * seg, e0), o);
}

// One block per segment (persistent over the segments), one thread per pixel
// of the segment's tile; splats staged RT_PIX at a time.  Writes the
// segment's (C, T) per pixel to part[seg][pixel].
__global__ void __launch_bounds__(RT_PIX) splat_segment_kernel(
    const uint4 *__restrict__ segs, const unsigned long long *__restrict__ n_segs_dev,
    const uint32_t *__restrict__ order, const float4 *__restrict__ payload, int W, int H,
    float4 *__restrict__ part) {
    __shared__ float4 s0[RT_PIX], s1[RT_PIX], s2[RT_PIX];
    const int ntx = (W + RT - 1) / RT, nty = (H + RT - 1) / RT;
    const unsigned long long n_segs = *n_segs_dev;
    for (unsigned long long sg = blockIdx.x; sg < n_segs; sg += gridDim.x) {
        const uint4 S = segs[sg];
        const int tile = (int)S.x;
        const int rem = tile % (ntx * nty), ti = rem / ntx, tj = rem - ti * ntx;
        const int i = ti * RT + threadIdx.x / RT, j = tj * RT + threadIdx.x % RT;
        const bool inside = i < H && j < W;
        const float px = (float)j + 0.5f, py = (float)i + 0.5f;
        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        bool done = !inside;
        for (uint32_t base = S.y; base < S.z; base += RT_PIX) {
            if (__syncthreads_count(done) == RT_PIX) break;
            const uint32_t e = base + threadIdx.x;
            if (e < S.z) {
                const uint32_t p = order[e];
                s0[threadIdx.x] = __ldg(payload + 3 * (size_t)p);
                s1[threadIdx.x] = __ldg(payload + 3 * (size_t)p + 1);
                s2[threadIdx.x] = __ldg(payload + 3 * (size_t)p + 2);
            }
            __syncthreads();
            const int cnt = (int)min((uint32_t)RT_PIX, S.z - base);
            for (int k = 0; k < cnt && !done; ++k) {
                const float4 a = s0[k], b = s1[k];
                const float m2 = splat_m2(px, py, a.x, a.y, a.z, a.w, b.x);
                if (!(m2 <= 9.0f)) continue;
                const float alpha = fminf(ALPHA_MAX, b.y * __expf(-0.5f * m2));
                const float4 c = s2[k];
                const float wgt = alpha * T;
                cr = fmaf(wgt, c.x, cr);
                cg = fmaf(wgt, c.y, cg);
                cb = fmaf(wgt, c.z, cb);
                T = T * (1.0f - alpha);
                if (T < T_CUT) done = true;
            }
        }
        __syncthreads();  // the staging buffers are refilled by the next segment
        part[sg * RT_PIX + threadIdx.x] = make_float4(cr, cg, cb, T);
    }
}

// Per pixel, the segments of its tile in order: C = C_0 + T_0 (C_1 + ...).
__global__ void splat_merge_kernel(const uint32_t *__restrict__ seg_cnt, const uint32_t *__restrict__ seg_off,
                                   const float4 *__restrict__ part, int64_t n_tiles, int W, int H,
                                   float *__restrict__ rgb) {
    const int ntx = (W + RT - 1) / RT, nty = (H + RT - 1) / RT;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_tiles * RT_PIX) return;
    const int64_t tile = gid / RT_PIX;
    const int px = (int)(gid - tile * RT_PIX);
    const int v = (int)(tile / (ntx * nty)), rem = (int)(tile - (int64_t)v * ntx * nty);
    const int ti = rem / ntx, tj = rem - ti * ntx;
    const int i = ti * RT + px / RT, j = tj * RT + px % RT;
    if (i >= H || j >= W) return;
    const uint32_t o = seg_off[tile], n = seg_cnt[tile];
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    for (uint32_t k = 0; k < n && T >= T_CUT; ++k) {
        const float4 q = part[(size_t)(o + k) * RT_PIX + px];
        cr = fmaf(T, q.x, cr);
        cg = fmaf(T, q.y, cg);
        cb = fmaf(T, q.z, cb);
        T *= q.w;
    }
    const size_t pix = ((size_t)v * H + i) * W + j;
    rgb[3 * pix] = cr;
    rgb[3 * pix + 1] = cg;
    rgb[3 * pix + 2] = cb;
}

// The six probe cameras at `centre`: rows U, V, F of each face, focal length
// and principal point face / 2 (a 90-degree field of view).
__global__ void cube_cams_kernel(const float *__restrict__ centre, int face, float *__restrict__ cams) {
    const int f = threadIdx.x;
    if (f >= 6) return;
    float *c = cams + CAM_F * f;
    for (int k = 0; k < 9; ++k) c[k] = 0.0f;
    c[0 + c_face_axis[f][1]] = c_face_sign[f][1];  // row x: U
    c[3 + c_face_axis[f][2]] = c_face_sign[f][2];  // row y: V
    c[6 + c_face_axis[f][0]] = c_face_sign[f][0];  // row forward: F
    c[9] = centre[0];
    c[10] = centre[1];
    c[11] = centre[2];
    const float fl = 0.5f * (float)face;
    c[12] = c[13] = c[14] = c[15] = fl;
}

// Texel-centre directions of the faces and their exact solid angles,
// w = omega(u1, v1) - omega(u0, v1) - omega(u1, v0) + omega(u0, v0) with
// omega(x, y) = atan2(x y, sqrt(x^2 + y^2 + 1)) (the integral of
// (1 + u^2 + v^2)^(-3/2) over [0, x] x [0, y]), in double precision.
__global__ void cube_dirs_kernel(int face, float *__restrict__ dirs, float *__restrict__ w) {
    const int64_t total = 6ll * face * face;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(p / ((int64_t)face * face));
        const int rem = (int)(p - (int64_t)f * face * face), i = rem / face, j = rem - i * face;
        const double u0 = 2.0 * j / face - 1.0, u1 = 2.0 * (j + 1) / face - 1.0;
        const double v0 = 2.0 * i / face - 1.0, v1 = 2.0 * (i + 1) / face - 1.0;
        auto om = [](double x, double y) { return atan2(x * y, sqrt(x * x + y * y + 1.0)); };
        w[p] = (float)(om(u1, v1) - om(u0, v1) - om(u1, v0) + om(u0, v0));
        const double u = 0.5 * (u0 + u1), v = 0.5 * (v0 + v1);
        double d[3];
        d[c_face_axis[f][0]] = c_face_sign[f][0];
        d[c_face_axis[f][1]] = c_face_sign[f][1] * u;
        d[c_face_axis[f][2]] = c_face_sign[f][2] * v;
        const double nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        dirs[3 * p] = (float)(d[0] / nrm);
        dirs[3 * p + 1] = (float)(d[1] / nrm);
        dirs[3 * p + 2] = (float)(d[2] / nrm);
    }
}

// The splatting pipeline for n_views cameras (device, CAM_F floats each) of
// W x H images; arguments checked, device current.
int render_impl(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats, const float *opac,
                const float *colors, int64_t n, const float *cams, int n_views, int W, int H, float near,
                float *rgb_out, int64_t *n_pairs_out, cudaStream_t s) {
    const int ntx = (W + RT - 1) / RT, nty = (H + RT - 1) / RT;
    const int64_t n_tiles = (int64_t)n_views * ntx * nty;
    int rc;
    const int64_t ns = n * n_views;  // splats
    void *w_rng;
    // per-tile [start, end), then the 8-byte pair and splat counters
    const size_t rng_bytes = (2 * sizeof(uint32_t) * (size_t)n_tiles + 7) & ~(size_t)7;
    if ((rc = ws_reserve(ctx, WS_RANGES, rng_bytes + 2 * sizeof(unsigned long long), &w_rng))) return rc;
    uint32_t *ts = (uint32_t *)w_rng, *te = ts + n_tiles;
    unsigned long long *d_total = (unsigned long long *)((char *)w_rng + rng_bytes);
    unsigned long long *d_ns = d_total + 1;
    cudaError_t e = cudaMemsetAsync(w_rng, 0, rng_bytes + 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "render: memset");
    uint64_t P = 0;
    const uint32_t *order = nullptr;     // splat of each sorted pair
    const float4 *payload = nullptr;     // per-splat payloads
    const int grid = (int)std::min<int64_t>((std::max<int64_t>(n, 1) + 255) / 256, (int64_t)ctx->num_sms * 16);
    uint32_t *sorder = nullptr, *soff = nullptr;
    const uint2 *rect = nullptr;
    if (n > 0) {
        // splats: depth keys and indices (sorted in place, with alternates),
        // tile counts (then their offsets in depth order), rectangles, payloads
        void *dk, *dv, *dk2, *dv2, *w_cnt, *w_spl;
        const size_t nsz = (size_t)ns;
        if ((rc = ws_reserve(ctx, WS_CKEYS_A, sizeof(uint32_t) * nsz, &dk))) return rc;
        if ((rc = ws_reserve(ctx, WS_CVALS_A, sizeof(uint32_t) * nsz, &dv))) return rc;
        if ((rc = ws_reserve(ctx, WS_CKEYS_B, sizeof(uint32_t) * nsz, &dk2))) return rc;
        if ((rc = ws_reserve(ctx, WS_CVALS_B, sizeof(uint32_t) * nsz, &dv2))) return rc;
        if ((rc = ws_reserve(ctx, WS_COUNTS, 2 * sizeof(uint32_t) * nsz, &w_cnt))) return rc;
        if ((rc = ws_reserve(ctx, WS_RENDER, (3 * sizeof(float4) + sizeof(uint2)) * nsz, &w_spl))) return rc;
        uint32_t *cnt = (uint32_t *)w_cnt;
        soff = cnt + nsz;
        float4 *pl = (float4 *)w_spl;
        uint2 *rc2 = (uint2 *)(pl + 3 * nsz);
        // keys by splat in dk, live flags in dk2 (then their scan); the live
        // splats' keys and indices compacted into dv2 and dv, sorted with dk
        // and dk2 as the alternates
        splat_prep_kernel<<<grid, 256, 0, s>>>(means, scales, quats, opac, colors, n, cams, n_views, W, H, near,
                                               (uint32_t *)dk, (uint32_t *)dk2, cnt, rc2, pl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "splat_prep_kernel");
        if ((rc = scan_exclusive_u32(ctx, (uint32_t *)dk2, (uint32_t *)dk2, ns, d_ns, s))) return rc;
        const int sgrid0 = (int)std::min<int64_t>((ns + 255) / 256, (int64_t)ctx->num_sms * 16);
        compact_splats_kernel<<<sgrid0, 256, 0, s>>>((const uint32_t *)dk, cnt, (const uint32_t *)dk2, ns,
                                                     (uint32_t *)dv2, (uint32_t *)dv);
        uint32_t *keys = (uint32_t *)dv2, *vals = (uint32_t *)dv;
        if ((rc = radix_sort_pairs(ctx, &keys, &vals, (uint32_t *)dk, (uint32_t *)dk2, d_ns, ns, 32, s)))
            return rc;
        sorder = vals;
        sorted_counts_kernel<<<sgrid0, 256, 0, s>>>(sorder, cnt, d_ns, ns, soff);
        if ((rc = scan_exclusive_u32(ctx, soff, soff, ns, d_total, s))) return rc;
        e = cudaMemcpyAsync(ctx->h_pinned, d_total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "render: pair count");
        P = ctx->h_pinned[0];
        if (P >= (1ull << 31)) return fail(ctx, DGSM_ERR_WORKSPACE, "render: more than 2^31 pairs");
        rect = rc2;
        payload = pl;
    }
    if (n_pairs_out) *n_pairs_out = (int64_t)P;
    if (P > 0) {
        void *ka, *va, *kb, *vb;
        if ((rc = ws_reserve(ctx, WS_KEYS_A, sizeof(uint32_t) * P, &ka))) return rc;
        if ((rc = ws_reserve(ctx, WS_VALS_A, sizeof(uint32_t) * P, &va))) return rc;
        if ((rc = ws_reserve(ctx, WS_KEYS_B, sizeof(uint32_t) * P, &kb))) return rc;
        if ((rc = ws_reserve(ctx, WS_VALS_B, sizeof(uint32_t) * P, &vb))) return rc;
        const int pgrid = (int)std::min<int64_t>((ns + PAIR_T - 1) / PAIR_T, (int64_t)ctx->num_sms * 64);
        splat_pairs_kernel<<<pgrid, PAIR_T, 0, s>>>(sorder, soff, rect, ns, d_ns, d_total, ntx, nty,
                                                    (uint32_t *)ka, (uint32_t *)va);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "splat_pairs_kernel");
        // (tile, splat) pairs in depth order, sorted stably by tile: every
        // tile's splats front to back
        uint32_t *tkeys = (uint32_t *)ka, *sids = (uint32_t *)va;
        int bits = 1;
        while (((int64_t)1 << bits) < n_tiles) ++bits;
        if ((rc = radix_sort_pairs(ctx, &tkeys, &sids, (uint32_t *)kb, (uint32_t *)vb, d_total, (int64_t)P, bits, s)))
            return rc;
        const int rgrid = (int)std::min<int64_t>(((int64_t)P + 255) / 256, (int64_t)ctx->num_sms * 16);
        splat_ranges_kernel<<<rgrid, 256, 0, s>>>(tkeys, d_total, ts, te);
        order = sids;
    }
    // segments of every tile's list (an empty tile has one empty segment):
    // long enough that a tile's front layers saturate within its first
    // segment, short enough that the segments give every SM 8 blocks
    const uint64_t fill = (uint64_t)ctx->num_sms * 8;
    const uint32_t seg = (uint32_t)std::max<uint64_t>(SEG_MIN, ((P + fill - 1) / fill + RT_PIX - 1) / RT_PIX * RT_PIX);
    const int64_t max_segs = (int64_t)(P / seg) + n_tiles;
    void *w_seg, *w_part;
    const size_t cnt_bytes = (sizeof(uint32_t) * (size_t)n_tiles + 15) & ~(size_t)15;
    if ((rc = ws_reserve(ctx, WS_SEGS, 2 * cnt_bytes + 16 + sizeof(uint4) * (size_t)max_segs, &w_seg))) return rc;
    if ((rc = ws_reserve(ctx, WS_PART, sizeof(float4) * RT_PIX * (size_t)max_segs, &w_part))) return rc;
    uint32_t *seg_cnt = (uint32_t *)w_seg, *seg_off = (uint32_t *)((char *)w_seg + cnt_bytes);
    unsigned long long *d_nseg = (unsigned long long *)((char *)w_seg + 2 * cnt_bytes);
    uint4 *segs = (uint4 *)((char *)w_seg + 2 * cnt_bytes + 16);
    const int tgrid = (int)((n_tiles + 255) / 256);
    seg_count_kernel<<<tgrid, 256, 0, s>>>(ts, te, n_tiles, seg, seg_cnt);
    if ((rc = scan_exclusive_u32(ctx, seg_cnt, seg_off, n_tiles, d_nseg, s))) return rc;
    seg_fill_kernel<<<tgrid, 256, 0, s>>>(ts, te, n_tiles, seg, seg_off, segs);
    // more blocks than fit at once, so the block scheduler balances segments of
    // different cost
    const int sgrid = (int)std::min<int64_t>(max_segs, (int64_t)ctx->num_sms * 64);
    splat_segment_kernel<<<sgrid, RT_PIX, 0, s>>>(segs, d_nseg, order, payload, W, H, (float4 *)w_part);
    splat_merge_kernel<<<(int)((n_tiles * RT_PIX + 255) / 256), 256, 0, s>>>(seg_cnt, seg_off, (const float4 *)w_part,
                                                                              n_tiles, W, H, rgb_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "splat render kernels");
}

int check_gaussians(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                    const float *opac, const float *colors, int64_t n, float near, const float *rgb_out) {
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: n out of range");
    if (n > 0 && (!means || !scales || !quats || !opac || !colors))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "render: null Gaussian array");
    if (!rgb_out) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: null output");
    if (!(near > 0.0f)) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: near must be > 0");
    return DGSM_OK;
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_cube_dirs(dgsm_ctx *ctx, int32_t face, float *dirs_out, float *w_out, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (face < 1 || face > 4096 || !dirs_out || !w_out)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "cube dirs: face in 1..4096 and output arrays required");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const int64_t total = 6ll * face * face;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8);
    cube_dirs_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(face, dirs_out, w_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "cube_dirs_kernel");
}

extern "C" int dgsm_render_views(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                                 const float *opac, const float *colors, int64_t n, const float *cams,
                                 int32_t n_views, int32_t W, int32_t H, float near, float *rgb_out,
                                 int64_t *n_pairs_out, void *stream) {
    DGSM_RANGE("dgsm_render_views");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    int rc = check_gaussians(ctx, means, scales, quats, opac, colors, n, near, rgb_out);
    if (rc) return rc;
    if (!cams || n_views < 1 || n_views > 64) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: need 1..64 cameras");
    if (n * n_views >= ((int64_t)1 << 32)) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: n x n_views >= 2^32");
    if (W < 1 || H < 1 || W > 4096 || H > 4096) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: W, H in 1..4096");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return render_impl(ctx, means, scales, quats, opac, colors, n, cams, n_views, W, H, near, rgb_out, n_pairs_out,
                       (cudaStream_t)stream);
}

extern "C" int dgsm_render_cubemap(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                                   const float *opac, const float *colors, int64_t n, const float *centre,
                                   int32_t face, float near, float *rgb_out, int64_t *n_pairs_out,
                                   void *stream) {
    DGSM_RANGE("dgsm_render_cubemap");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    int rc = check_gaussians(ctx, means, scales, quats, opac, colors, n, near, rgb_out);
    if (rc) return rc;
    if (!centre) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: null centre");
    if (n * 6 >= ((int64_t)1 << 32)) return fail(ctx, DGSM_ERR_INVALID_ARG, "render: 6 n >= 2^32");
    if (face < RT || face > 1024 || face % RT != 0)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "render: face must be a multiple of 8 in 8..1024");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    void *w_cams;
    if ((rc = ws_reserve(ctx, WS_CAMS, 6 * CAM_F * sizeof(float), &w_cams))) return rc;
    cube_cams_kernel<<<1, 32, 0, s>>>(centre, face, (float *)w_cams);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cube_cams_kernel");
    return render_impl(ctx, means, scales, quats, opac, colors, n, (const float *)w_cams, 6, face, face, near,
                       rgb_out, n_pairs_out, s);
}
