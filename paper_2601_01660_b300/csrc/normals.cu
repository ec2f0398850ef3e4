// normals.cu -- pseudo-normals of Gaussians by local PCA (Sec. 4, lighting
// consistency): for Gaussian i, the Gaussians j within radius r of its
// centre, weighted w_j = alpha_j (1 - |x_j - x_i|^2 / r^2)^2; the unit
// eigenvector of the smallest eigenvalue of their weighted covariance; the
// smallest-scale axis when fewer than three neighbours carry weight or the
// covariance vanishes; turned away from a reference point.
//
// Neighbour search: a spatial hash of cells of edge r.  The Gaussians are
// sorted by bucket (stable radix sort, so each bucket lists its Gaussians in
// index order and the sums below have a fixed order), their (x, y, z, alpha)
// gathered in that order, and each thread walks the 27 cells around its
// Gaussian's cell; a candidate counts only in its own cell, so a bucket that
// two of the 27 cells share is never counted twice.
#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int NRM_THREADS = 256;
constexpr int JACOBI_SWEEPS = 6;

struct Cell {
    int x, y, z;
};

// Cell of a point: floor(p / r) per axis, clamped to +-2^24 (beyond that the
// floats are too coarse for cells of this size anyway).
__device__ __forceinline__ Cell cell_of(float x, float y, float z, float inv_r) {
    const float lim = 16777216.0f;
    Cell c;
    c.x = (int)fminf(fmaxf(floorf(__fmul_rn(x, inv_r)), -lim), lim);
    c.y = (int)fminf(fmaxf(floorf(__fmul_rn(y, inv_r)), -lim), lim);
    c.z = (int)fminf(fmaxf(floorf(__fmul_rn(z, inv_r)), -lim), lim);
    return c;
}

// Bucket of a cell: the three coordinates mixed by large odd multipliers,
// then a multiplicative hash keeping the top `bits` bits.
__device__ __forceinline__ uint32_t cell_bucket(Cell c, int bits) {
    const uint32_t h = ((uint32_t)c.x * 73856093u) ^ ((uint32_t)c.y * 19349663u) ^ ((uint32_t)c.z * 83492791u);
    return (h * 2654435761u) >> (32 - bits);
}

__global__ void nrm_count_kernel(int64_t n, unsigned long long *__restrict__ d_n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_n = (unsigned long long)n;
}

__global__ void nrm_key_kernel(const float *__restrict__ means, int64_t n, float inv_r, int bits,
                               uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Cell c = cell_of(means[3 * i], means[3 * i + 1], means[3 * i + 2], inv_r);
    keys[i] = cell_bucket(c, bits);
    vals[i] = (uint32_t)i;
}

// start/end of every non-empty bucket in the sorted order (the arrays are
// zeroed first, so an empty bucket reads [0, 0)).
__global__ void nrm_ranges_kernel(const uint32_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ start,
                                  uint32_t *__restrict__ end) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t k = keys[p];
    if (p == 0 || keys[p - 1] != k) start[k] = (uint32_t)p;
    if (p == n - 1 || keys[p + 1] != k) end[k] = (uint32_t)(p + 1);
}

__global__ void nrm_gather_kernel(const float *__restrict__ means, const float *__restrict__ opac,
                                  const uint32_t *__restrict__ vals, int64_t n, float4 *__restrict__ pts) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t i = vals[p];
    pts[p] = make_float4(means[3 * i], means[3 * i + 1], means[3 * i + 2], opac[i]);
}

// Eigen-decomposition of the symmetric 3x3 matrix a (a00 a01 a02 a11 a12
// a22) by cyclic Jacobi rotations (each rotation zeroes one off-diagonal
// entry with the smaller of the two angles, t = sgn(theta) / (|theta| +
// sqrt(theta^2 + 1)), theta = (a_qq - a_pp) / (2 a_pq)); returns the unit
// eigenvector of the smallest eigenvalue (first on ties).
__device__ __forceinline__ void smallest_eigvec(float a00, float a01, float a02, float a11, float a12, float a22, float *v) {
    float A[3][3] = {{a00, a01, a02}, {a01, a11, a12}, {a02, a12, a22}};
    float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
#pragma unroll
    for (int sweep = 0; sweep < JACOBI_SWEEPS; ++sweep) {
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const float apq = A[p][q];
            if (fabsf(apq) <= 1e-30f) continue;
            const float theta = (A[q][q] - A[p][p]) / (2.0f * apq);
            const float t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
            const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c;
            // A <- J^T A J with J the rotation in the (p, q) plane
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
    // column of the smallest diagonal entry, chosen by selects (no indexed
    // register arrays)
    float lo = A[0][0], x = V[0][0], y = V[1][0], z = V[2][0];
    if (A[1][1] < lo) { lo = A[1][1]; x = V[0][1]; y = V[1][1]; z = V[2][1]; }
    if (A[2][2] < lo) { x = V[0][2]; y = V[1][2]; z = V[2][2]; }
    const float inv = rsqrtf(x * x + y * y + z * z);
    v[0] = x * inv;
    v[1] = y * inv;
    v[2] = z * inv;
}

// Smallest-scale axis (first on ties) of the rotation of quaternion q
// (w, x, y, z): a column of R.
__device__ __forceinline__ void smallest_axis(float4 q, float sx, float sy, float sz, float *v) {
    const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    int k = 0;
    float sm = sx;
    if (sy < sm) { k = 1; sm = sy; }
    if (sz < sm) k = 2;
    if (k == 0) {
        v[0] = 1.0f - 2.0f * (y * y + z * z); v[1] = 2.0f * (x * y + w * z); v[2] = 2.0f * (x * z - w * y);
    } else if (k == 1) {
        v[0] = 2.0f * (x * y - w * z); v[1] = 1.0f - 2.0f * (x * x + z * z); v[2] = 2.0f * (y * z + w * x);
    } else {
        v[0] = 2.0f * (x * z + w * y); v[1] = 2.0f * (y * z - w * x); v[2] = 1.0f - 2.0f * (x * x + y * y);
    }
}

// G lanes per Gaussian (G divides 32), Gaussians in bucket order so that
// neighbouring groups walk the same cells; the lanes of a group split every
// bucket's candidates and combine their sums by shuffles, then the group's
// first lane solves the 3x3 problem.  Offsets are taken in units of r, so
// the covariance is O(1).
template <int G>
__global__ void __launch_bounds__(NRM_THREADS) nrm_pca_kernel(
    const float4 *__restrict__ pts, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ bstart,
    const uint32_t *__restrict__ bend, int64_t n, float inv_r, int bits, const float4 *__restrict__ quats,
    const float *__restrict__ scales, const float *__restrict__ centroid, float *__restrict__ normals) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int sub = (int)(threadIdx.x & (G - 1));
    const bool live = p < n;  // lanes past the end still take part in the shuffles
    const float4 me = live ? pts[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    const Cell c0 = cell_of(me.x, me.y, me.z, inv_r);
    float W = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
    float s00 = 0.f, s01 = 0.f, s02 = 0.f, s11 = 0.f, s12 = 0.f, s22 = 0.f;
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const Cell cc = {c0.x + dx, c0.y + dy, c0.z + dz};
                const uint32_t b = cell_bucket(cc, bits);
                const uint32_t e1 = live ? bend[b] : 0u;
                for (uint32_t q = (live ? bstart[b] : 0u) + sub; q < e1; q += G) {
                    const float4 o = pts[q];
                    const Cell co = cell_of(o.x, o.y, o.z, inv_r);
                    if (co.x != cc.x || co.y != cc.y || co.z != cc.z) continue;  // another cell of this bucket
                    const float ux = (o.x - me.x) * inv_r, uy = (o.y - me.y) * inv_r, uz = (o.z - me.z) * inv_r;
                    const float d2 = ux * ux + uy * uy + uz * uz;
                    if (!(d2 <= 1.0f)) continue;
                    const float t = 1.0f - d2;
                    const float w = o.w * t * t;
                    if (!(w > 0.0f)) continue;
                    ++cnt;
                    W += w;
                    m0 = fmaf(w, ux, m0); m1 = fmaf(w, uy, m1); m2 = fmaf(w, uz, m2);
                    s00 = fmaf(w * ux, ux, s00); s01 = fmaf(w * ux, uy, s01); s02 = fmaf(w * ux, uz, s02);
                    s11 = fmaf(w * uy, uy, s11); s12 = fmaf(w * uy, uz, s12); s22 = fmaf(w * uz, uz, s22);
                }
            }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        W += __shfl_xor_sync(0xffffffffu, W, o);
        m0 += __shfl_xor_sync(0xffffffffu, m0, o);
        m1 += __shfl_xor_sync(0xffffffffu, m1, o);
        m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        s00 += __shfl_xor_sync(0xffffffffu, s00, o);
        s01 += __shfl_xor_sync(0xffffffffu, s01, o);
        s02 += __shfl_xor_sync(0xffffffffu, s02, o);
        s11 += __shfl_xor_sync(0xffffffffu, s11, o);
        s12 += __shfl_xor_sync(0xffffffffu, s12, o);
        s22 += __shfl_xor_sync(0xffffffffu, s22, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (!live || sub != 0) return;
    const uint32_t i = vals[p];
    float v[3];
    bool pca = cnt >= 3 && W > 0.0f;
    if (pca) {
        const float iw = 1.0f / W;
        m0 *= iw; m1 *= iw; m2 *= iw;
        const float c00 = s00 * iw - m0 * m0, c01 = s01 * iw - m0 * m1, c02 = s02 * iw - m0 * m2;
        const float c11 = s11 * iw - m1 * m1, c12 = s12 * iw - m1 * m2, c22 = s22 * iw - m2 * m2;
        pca = c00 + c11 + c22 > 0.0f;
        if (pca) smallest_eigvec(c00, c01, c02, c11, c12, c22, v);
    }
    if (!pca) smallest_axis(quats[i], scales[3 * i], scales[3 * i + 1], scales[3 * i + 2], v);
    const float side = v[0] * (me.x - centroid[0]) + v[1] * (me.y - centroid[1]) + v[2] * (me.z - centroid[2]);
    const float sg = side < 0.0f ? -1.0f : 1.0f;
    normals[3 * i] = sg * v[0];
    normals[3 * i + 1] = sg * v[1];
    normals[3 * i + 2] = sg * v[2];
}

// Lanes per Gaussian: more for fewer Gaussians, so that small sets (one
// avatar) still fill the GPU (measured on B300: 100k avatar Gaussians 0.95,
// 0.76, 0.69 ms with 2, 4, 8 lanes; the 1.6M room 2.18, 2.02, 2.25 ms).
inline int nrm_lanes(int64_t n) { return n <= (1 << 18) ? 8 : 4; }

template <int G>
void launch_nrm_pca(int64_t n, cudaStream_t s, const float4 *pts, const uint32_t *vals, const uint32_t *bstart,
                    const uint32_t *bend, float inv_r, int bits, const float4 *quats, const float *scales,
                    const float *centroid, float *normals) {
    const unsigned grid = (unsigned)((n * G + NRM_THREADS - 1) / NRM_THREADS);
    nrm_pca_kernel<G><<<grid, NRM_THREADS, 0, s>>>(pts, vals, bstart, bend, n, inv_r, bits, quats, scales,
                                                   centroid, normals);
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int dgsm_pca_normals(dgsm_ctx *ctx, const float *means, const float *opac, const float *quats,
                                const float *scales, int64_t n, float radius, const float *centroid,
                                float *normals_out, void *stream) {
    DGSM_RANGE("dgsm_pca_normals");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || n > 0x7fffffffLL) return fail(ctx, DGSM_ERR_INVALID_ARG, "pca normals: 0 <= n < 2^31");
    if (!(radius > 0.0f) || !(radius < INFINITY))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "pca normals: radius must be positive and finite");
    if (n == 0) return DGSM_OK;
    if (!means || !opac || !quats || !scales || !centroid || !normals_out)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "pca normals: null array");
    if (((uintptr_t)quats & 15u) != 0) return fail(ctx, DGSM_ERR_INVALID_ARG, "pca normals: quats not 16-byte aligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const cudaStream_t s = (cudaStream_t)stream;
    // 2^bits buckets, at least twice the Gaussians (few collisions), at most 2^30
    int bits = 10;
    while (bits < 30 && (1LL << bits) < 2 * n) ++bits;
    const size_t nb = (size_t)1 << bits, nn = (size_t)n;
    const size_t off_keys = 0, off_vals = off_keys + 4 * nn, off_keys2 = off_vals + 4 * nn,
                 off_vals2 = off_keys2 + 4 * nn, off_start = off_vals2 + 4 * nn, off_end = off_start + 4 * nb,
                 off_cnt = (off_end + 4 * nb + 15) & ~(size_t)15, off_pts = off_cnt + 16,
                 total = off_pts + 16 * nn;
    void *w;
    int rc = ws_reserve(ctx, WS_NORMALS, total, &w);
    if (rc) return rc;
    char *base = (char *)w;
    uint32_t *keys = (uint32_t *)(base + off_keys), *vals = (uint32_t *)(base + off_vals);
    uint32_t *keys2 = (uint32_t *)(base + off_keys2), *vals2 = (uint32_t *)(base + off_vals2);
    uint32_t *bstart = (uint32_t *)(base + off_start), *bend = (uint32_t *)(base + off_end);
    unsigned long long *d_n = (unsigned long long *)(base + off_cnt);
    float4 *pts = (float4 *)(base + off_pts);
    const float inv_r = 1.0f / radius;
    const unsigned grid = (unsigned)((n + NRM_THREADS - 1) / NRM_THREADS);
    nrm_count_kernel<<<1, 32, 0, s>>>(n, d_n);
    nrm_key_kernel<<<grid, NRM_THREADS, 0, s>>>(means, n, inv_r, bits, keys, vals);
    rc = radix_sort_pairs(ctx, &keys, &vals, keys2, vals2, d_n, n, bits, s);
    if (rc) return rc;
    e = cudaMemsetAsync(bstart, 0, 8 * nb, s);  // bstart and bend are adjacent
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pca normals: memset");
    nrm_ranges_kernel<<<grid, NRM_THREADS, 0, s>>>(keys, n, bstart, bend);
    nrm_gather_kernel<<<grid, NRM_THREADS, 0, s>>>(means, opac, vals, n, pts);
    const float4 *q4 = reinterpret_cast<const float4 *>(quats);
    switch (nrm_lanes(n)) {
        case 8: launch_nrm_pca<8>(n, s, pts, vals, bstart, bend, inv_r, bits, q4, scales, centroid, normals_out); break;
        default: launch_nrm_pca<4>(n, s, pts, vals, bstart, bend, inv_r, bits, q4, scales, centroid, normals_out);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "pca normals kernels");
}
