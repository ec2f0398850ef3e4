// dgsm_internal.cuh -- shared declarations of libdgsm.so (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dgsm.h"

// ---------------------------------------------------------------------------
// Context: device, error text, device status word, growable workspace.
// ---------------------------------------------------------------------------
enum WsSlot {
    WS_BUILD_REC = 0,  // per (light, Gaussian) build record, 80 B
    WS_BIN_REC,        // per (light, Gaussian) binning record, 80 B
    WS_COUNTS,         // per (light, Gaussian) super-tile count / offset, u32
    WS_SCAN_TMP,       // scan block sums
    WS_CONES,          // tile + super-tile cones
    WS_KEYS_A, WS_VALS_A, WS_KEYS_B, WS_VALS_B,
    WS_HIST,           // radix histograms (+ their scan)
    WS_RANGES,         // per (light, tile) start/end
    WS_ITEMS,          // build work items (+ per-key item counts, item counter)
    WS_ACCUM,          // per-voxel tau accumulators of tiles split into several items
    WS_DONE,           // per-key count of finished items
    WS_SH_PART,        // SH fit per-block partial sums
    WS_CENTROID,       // weighted-centroid partial sums
    WS_FRAME,          // device copies of a host frame (dgsm_frame_host)
    WS_NF,             // surrogate training: per-sample rows and partial gradients
    WS_NF_ACC,         // surrogate attenuation over more than four lights: partial sums
    WS_POSES,          // rigid poses of moving objects, copied in per call
    WS_CKEYS_A, WS_CVALS_A, WS_CKEYS_B, WS_CVALS_B,  // (super-tile, Gaussian) pairs
    WS_CRANGES,        // per (light, super-tile) start/end of its Gaussian list
    WS_UNITS,          // fine-binning work units (+ per-super-tile unit counts)
    WS_FCNT, WS_FOFF,  // per (unit, tile) pair counts and their scan
    WS_FMASK,          // per (unit, tile) bitmaps of the Gaussians that reach it (and its halves)
    WS_ROI,            // region of interest: shell ranges, texel mask, tile and super-tile flags
    WS_RENDER,         // splat render: per-pair splat payloads
    WS_CAMS,           // the six probe cameras of dgsm_render_cubemap
    WS_SEGS,           // splat render: per-tile segment counts and offsets, the segments
    WS_PART,           // splat render: per-segment partial colour and transmittance of each pixel
    WS_NORMALS,        // pca normals: bucket keys and order, bucket ranges, sorted points
    WS_PFRAME,         // persistent frame kernel: control words, binning, items, records
    WS_PF_CONES,       // persistent frame kernel: the dynamic atlas's tile cones
    WS_PF_PHASE,       // persistent frame kernel: phase timestamps (while profiling)
    WS_SMASK,          // build: per (light, Gaussian) mask of the super-tiles it reaches
    WS_KCNT,           // build: per (light, super-tile) pair counts and cursors
    WS_ORDER,          // spatial order: Z-order keys and indices, the bounding box
    WS_FQ0, WS_FQ1,    // pipelined host frames: each slot's device copies of its frame
    WS_NSLOTS
};

struct dgsm_ctx {
    int device = 0;
    std::string err;
    void *ws[WS_NSLOTS] = {};
    size_t ws_cap[WS_NSLOTS] = {};
    int *d_status = nullptr;                 // first error code recorded by a kernel
    // [0] rays tested, [1] ray evals, [2] shell evals, [3] binned pairs,
    // [4] pairs the build keeps (= [3], or 0 when they overflow max_pairs)
    unsigned long long *d_stats = nullptr;
    unsigned long long *h_pinned = nullptr;  // pinned staging for small device->host reads
    int num_sms = 148;
    // optional phase timing of dgsm_build: events recorded on the caller's stream
    static constexpr int PROF_RING = 256;
    bool prof = false;
    int prof_count = 0;
    cudaEvent_t prof_ev[PROF_RING][3] = {};
    // > 0 while a graph captured on this context is alive: its nodes hold
    // workspace addresses, so the workspace must not move
    int frozen = 0;
    // side stream and events of dgsm_frame_host (copies beside compute)
    cudaStream_t side = nullptr;
    cudaEvent_t fev[4] = {};
    // pipelined host frames (dgsm_frame_host_submit / _wait): two copy-in
    // streams, one copy-out stream, per slot six events, a pinned status word
    // and whether a frame is in flight
    cudaStream_t fq_h2d[2] = {}, fq_d2h = nullptr;
    cudaEvent_t fq_ev[2][6] = {};
    int *fq_status = nullptr;
    bool fq_busy[2] = {};
    // tile cones of the persistent frame kernel: valid for this buffer and atlas size
    void *pf_cones = nullptr;
    int pf_cones_h = 0, pf_cones_w = 0;
};

#include <nvtx3/nvToolsExt.h>

namespace dgsm {

// Contiguous objects of a Gaussian array (avatars): object o holds the
// Gaussians [s[o], s[o+1]).  Passed to kernels by value, so a captured graph
// keeps it.
constexpr int MAX_OBJECTS = 64;
struct Segs {
    long long s[MAX_OBJECTS + 1];
    int n;
};
// Host check: 1 <= n_obj <= MAX_OBJECTS, seg[0] = 0, nondecreasing, seg[n_obj] = n.
bool make_segs(const int64_t *seg, int n_obj, int64_t n, Segs *out);

// Records the first error code a kernel meets in the context's status word.
__device__ __forceinline__ void record_status(int *status, int code) { atomicCAS(status, 0, code); }

// Object holding Gaussian g (s[0] <= g < s[n]): the last o with s[o] <= g.
__device__ __forceinline__ int seg_find(const Segs &sg, long long g) {
    int lo = 0, hi = sg.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sg.s[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// An NVTX range around a library call (header-only NVTX: a no-op unless a
// profiler is attached), so that profiles can be cut by entry point.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define DGSM_RANGE(name) ::dgsm::NvtxRange dgsm_nvtx_range_(name)

int fail(dgsm_ctx *ctx, int code, const std::string &msg);
int cuda_fail(dgsm_ctx *ctx, cudaError_t e, const char *what);
// Ensures workspace slot `slot` holds at least `bytes`; may synchronise the device.
int ws_reserve(dgsm_ctx *ctx, int slot, size_t bytes, void **out);

// Device-wide exclusive scan of n uint32 values (in may equal out).  Writes
// the 64-bit total to *d_total (device).  Needs ctx workspace WS_SCAN_TMP.
int scan_exclusive_u32(dgsm_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n,
                       unsigned long long *d_total, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// The pair count is read on the device from *d_n (at most n_max, which
// sizes the launches).  Sorted result ends in (*keys_io, *vals_io) (the
// pointers may be swapped with the alternate buffers).
int radix_sort_pairs(dgsm_ctx *ctx, uint32_t **keys_io, uint32_t **vals_io, uint32_t *keys_alt,
                     uint32_t *vals_alt, const unsigned long long *d_n, int64_t n_max, int bits,
                     cudaStream_t s);

// ---------------------------------------------------------------------------
// IEEE single-precision operations that are never contracted or reordered:
// every integer decision of the octahedral index and of the tile binning is
// taken with these so that it is reproducible bit for bit on the CPU.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float xdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float xsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float sgn_pos(float x) { return x >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ float xdot(float ax, float ay, float az, float bx, float by, float bz) {
    return xadd(xadd(xmul(ax, bx), xmul(ay, by)), xmul(az, bz));
}

// Texel-centre coordinate (2j+1)/W - 1.
__device__ __forceinline__ float xcentre(int j, int W) {
    return xsub(xdiv((float)(2 * j + 1), (float)W), 1.0f);
}

// Octahedral decode (inverse of Eq. 6): undo the fold, z = 1-|u|-|v|, normalise.
__device__ __forceinline__ float3 xdecode(float u, float v) {
    float au = fabsf(u), av = fabsf(v);
    float z = xsub(xsub(1.0f, au), av);
    float x = u, y = v;
    if (z < 0.0f) {
        x = xmul(sgn_pos(u), xsub(1.0f, av));
        y = xmul(sgn_pos(v), xsub(1.0f, au));
    }
    float n = xsqrt(xadd(xadd(xmul(x, x), xmul(y, y)), xmul(z, z)));
    return make_float3(xdiv(x, n), xdiv(y, n), xdiv(z, n));
}

// Octahedral encode (Eq. 6) of the un-normalised vector v: q = v / |v|_1.
__device__ __forceinline__ float2 xencode(float vx, float vy, float vz) {
    float s = xadd(xadd(fabsf(vx), fabsf(vy)), fabsf(vz));
    if (s == 0.0f) return make_float2(0.0f, 0.0f);
    float qx = xdiv(vx, s), qy = xdiv(vy, s);
    if (vz >= 0.0f) return make_float2(qx, qy);
    return make_float2(xmul(sgn_pos(qx), xsub(1.0f, fabsf(qy))),
                       xmul(sgn_pos(qy), xsub(1.0f, fabsf(qx))));
}

// Cube-map atlas (the alternative parameterisation of the paper's ablation
// (C)): six F x F faces stacked as rows [f F, (f+1) F) of an atlas with
// H = 6F, W = F.  Face f has forward axis F_f and texel axes U_f (columns,
// u) and V_f (rows, v) as signed unit axes; texel (u, v) looks along
// F_f + u U_f + v V_f: (+x, -z, -y), (-x, +z, -y), (+y, +x, +z), (-y, +x, -z),
// (+z, +x, -y), (-z, -x, -y) (the usual cube-map faces).
enum { MAP_OCTA = 0, MAP_CUBE = 1 };

__device__ __forceinline__ void cube_axes(int f, int &aF, int &aU, int &aV, float &sF, float &sU, float &sV) {
    switch (f) {
        case 0: aF = 0; aU = 2; aV = 1; sF = 1.f; sU = -1.f; sV = -1.f; break;
        case 1: aF = 0; aU = 2; aV = 1; sF = -1.f; sU = 1.f; sV = -1.f; break;
        case 2: aF = 1; aU = 0; aV = 2; sF = 1.f; sU = 1.f; sV = 1.f; break;
        case 3: aF = 1; aU = 0; aV = 2; sF = -1.f; sU = 1.f; sV = -1.f; break;
        case 4: aF = 2; aU = 0; aV = 1; sF = 1.f; sU = 1.f; sV = -1.f; break;
        default: aF = 2; aU = 0; aV = 1; sF = -1.f; sU = -1.f; sV = -1.f; break;
    }
}

__device__ __forceinline__ float pick3(float x, float y, float z, int a) { return a == 0 ? x : a == 1 ? y : z; }

// Unit direction of the point (u, v) of cube face f.
__device__ __forceinline__ float3 xdecode_cube(int f, float u, float v) {
    int aF, aU, aV;
    float sF, sU, sV;
    cube_axes(f, aF, aU, aV, sF, sU, sV);
    const float cF = sF, cU = sU * u, cV = sV * v;  // sign flips: exact
    const float x = aF == 0 ? cF : aU == 0 ? cU : cV;
    const float y = aF == 1 ? cF : aU == 1 ? cU : cV;
    const float z = aF == 2 ? cF : aU == 2 ? cU : cV;
    const float n = xsqrt(xadd(xadd(xmul(x, x), xmul(y, y)), xmul(z, z)));
    return make_float3(xdiv(x, n), xdiv(y, n), xdiv(z, n));
}

// Cube encode of the un-normalised vector v: the face of the largest
// component (ties go to x, then y; a component >= 0 picks the positive face)
// and the face coordinates u = U.v / m, v = V.v / m, m that component's size.
__device__ __forceinline__ int xencode_cube(float vx, float vy, float vz, float &u, float &v) {
    const float ax = fabsf(vx), ay = fabsf(vy), az = fabsf(vz);
    const int f = (ax >= ay && ax >= az) ? (vx >= 0.0f ? 0 : 1) : (ay >= az ? (vy >= 0.0f ? 2 : 3) : (vz >= 0.0f ? 4 : 5));
    int aF, aU, aV;
    float sF, sU, sV;
    cube_axes(f, aF, aU, aV, sF, sU, sV);
    const float m = fabsf(pick3(vx, vy, vz, aF));
    if (m == 0.0f) {
        u = v = 0.0f;
        return f;
    }
    u = xdiv(sU * pick3(vx, vy, vz, aU), m);
    v = xdiv(sV * pick3(vx, vy, vz, aV), m);
    return f;
}

// Index decisions of one lookup (shared by attenuate and sample_index).
struct SampleIndex {
    int ci, cj;    // texel cell containing the point
    int bi, bj;    // bilinear base tap (may be -1 or H-1/W-1 before clamping)
    int r0, hf;    // rows of the point's face: [r0, r0 + hf) (0, H for the octahedral map)
    int k;         // #{radii <= t} - 1
    float fy, fx;  // bilinear fractions
    float t;       // distance to the light
};

__device__ __forceinline__ int count_le(const float *r, int K, float t) {
    // number of radii <= t (radii strictly increasing)
    int lo = 0, hi = K;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (r[mid] <= t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// A per-block guess table for the shell index: tab[b] = #{radii <= t_b} - 1
// at the start t_b of bin b of SHELL_BINS equal bins of log2 t over
// [radii[0], radii[K-1]].  shell_index() starts from the guess and steps to
// the exact comparison count, so the result equals count_le(t) - 1 whatever
// the radii (the table only saves the search).
constexpr int SHELL_BINS = 256;

struct ShellTab {
    float lr0, scale;  // log2 radii[0] and bins per unit of log2 t (0: no table)
};

// Fill tab (SHELL_BINS shorts in shared memory) from the block's radii rs;
// all threads of the block call it; a __syncthreads() must follow.
__device__ __forceinline__ ShellTab build_shell_tab(const float *rs, int K, short *tab) {
    ShellTab st;
    st.lr0 = 0.0f;
    st.scale = 0.0f;
    if (K >= 2 && rs[0] > 0.0f && rs[K - 1] > rs[0]) {
        st.lr0 = __log2f(rs[0]);
        st.scale = (float)SHELL_BINS / (__log2f(rs[K - 1]) - st.lr0);
    }
    for (int b = threadIdx.x; b < SHELL_BINS; b += blockDim.x) {
        const float tb = st.scale > 0.0f ? exp2f(st.lr0 + (float)b / st.scale) : rs[0];
        tab[b] = (short)max(count_le(rs, K, tb) - 1, 0);
    }
    return st;
}

__device__ __forceinline__ int shell_index(float t, const float *rs, int K, const short *tab, ShellTab st) {
    if (!(t >= rs[0])) return -1;
    if (t >= rs[K - 1]) return K - 1;
    const int b = min(max((int)((__log2f(t) - st.lr0) * st.scale), 0), SHELL_BINS - 1);
    int k = tab[b];
    while (k + 1 < K && rs[k + 1] <= t) ++k;
    while (k >= 0 && rs[k] > t) --k;
    return k;
}

// sample_index with the shell index from a guess table (same result).
__device__ __forceinline__ SampleIndex sample_index_tab(float px, float py, float pz, float ox, float oy,
                                                        float oz, int H, int W, const float *radii, int K,
                                                        const short *tab, ShellTab st) {
    SampleIndex s;
    float vx = xsub(px, ox), vy = xsub(py, oy), vz = xsub(pz, oz);
    s.t = xsqrt(xadd(xadd(xmul(vx, vx), xmul(vy, vy)), xmul(vz, vz)));
    float2 uv = xencode(vx, vy, vz);
    float fu = xmul(xmul(xadd(uv.x, 1.0f), 0.5f), (float)W);
    float fv = xmul(xmul(xadd(uv.y, 1.0f), 0.5f), (float)H);
    float gx = xsub(fu, 0.5f), gy = xsub(fv, 0.5f);
    float bj = floorf(gx), bi = floorf(gy);
    s.cj = min(max((int)floorf(fu), 0), W - 1);
    s.ci = min(max((int)floorf(fv), 0), H - 1);
    s.bj = (int)bj;
    s.bi = (int)bi;
    s.fx = xsub(gx, bj);
    s.fy = xsub(gy, bi);
    s.r0 = 0;
    s.hf = H;
    s.k = shell_index(s.t, radii, K, tab, st);
    return s;
}

__device__ __forceinline__ SampleIndex sample_index(float px, float py, float pz, float ox,
                                                    float oy, float oz, int H, int W,
                                                    const float *radii, int K) {
    SampleIndex s;
    float vx = xsub(px, ox), vy = xsub(py, oy), vz = xsub(pz, oz);
    s.t = xsqrt(xadd(xadd(xmul(vx, vx), xmul(vy, vy)), xmul(vz, vz)));
    float2 uv = xencode(vx, vy, vz);
    float fu = xmul(xmul(xadd(uv.x, 1.0f), 0.5f), (float)W);
    float fv = xmul(xmul(xadd(uv.y, 1.0f), 0.5f), (float)H);
    float gx = xsub(fu, 0.5f), gy = xsub(fv, 0.5f);
    float bj = floorf(gx), bi = floorf(gy);
    s.cj = min(max((int)floorf(fu), 0), W - 1);
    s.ci = min(max((int)floorf(fv), 0), H - 1);
    s.bj = (int)bj;
    s.bi = (int)bi;
    s.fx = xsub(gx, bj);
    s.fy = xsub(gy, bi);
    s.r0 = 0;
    s.hf = H;
    s.k = count_le(radii, K, s.t) - 1;
    return s;
}

// The same decisions on a cube-map atlas of F x F faces (H = 6F, W = F):
// rows are global (face f's rows start at f F); the bilinear taps are
// clamped to the point's face.  tab (or nullptr: a comparison count) as for
// sample_index_tab.
__device__ __forceinline__ SampleIndex sample_index_cube(float px, float py, float pz, float ox, float oy,
                                                         float oz, int F, const float *radii, int K,
                                                         const short *tab, ShellTab st) {
    SampleIndex s;
    float vx = xsub(px, ox), vy = xsub(py, oy), vz = xsub(pz, oz);
    s.t = xsqrt(xadd(xadd(xmul(vx, vx), xmul(vy, vy)), xmul(vz, vz)));
    float u, v;
    const int f = xencode_cube(vx, vy, vz, u, v);
    float fu = xmul(xmul(xadd(u, 1.0f), 0.5f), (float)F);
    float fv = xmul(xmul(xadd(v, 1.0f), 0.5f), (float)F);
    float gx = xsub(fu, 0.5f), gy = xsub(fv, 0.5f);
    float bj = floorf(gx), bi = floorf(gy);
    s.r0 = f * F;
    s.hf = F;
    s.cj = min(max((int)floorf(fu), 0), F - 1);
    s.ci = s.r0 + min(max((int)floorf(fv), 0), F - 1);
    s.bj = (int)bj;
    s.bi = s.r0 + (int)bi;
    s.fx = xsub(gx, bj);
    s.fy = xsub(gy, bi);
    s.k = tab ? shell_index(s.t, radii, K, tab, st) : count_le(radii, K, s.t) - 1;
    return s;
}

}  // namespace dgsm
