// nf.cu -- learned transmittance surrogate: a per-light neural field that
// stands in for the static-scene atlas lookup of Sec. 3.3.
//
// Field: T_hat(u, v, rho) = sigmoid(w5 . h4 + b5), h_l = ReLU(W_l h_{l-1} + b_l)
// (four hidden layers of width 64), h_0 = 96 Fourier features
// sin/cos(pi f_m x), f_m = 2^(8m/15) as float32, m = 0..15, of x in {u, v, rho}:
// u, v the octahedral coordinates of the direction (Eq. 6), rho the
// fractional shell coordinate in [0, 1].  Features, weights and hidden
// activations are bfloat16, sums and biases float32.
//
// Training (on atlases built by dgsm_build): voxels drawn at random, MSE on T,
// Adam; forward/backward per sample in FP32 SIMT (nf_fwdbwd_kernel), weight
// gradients as a batch reduction (nf_wgrad_kernel), Adam (nf_adam_kernel).
// Inference: bf16 tensor-core MMA (mma.sync m16n8k16, FP32 accumulate), the
// output fragments of one layer re-packed in registers as the input
// fragments of the next (nf_infer_kernel, nf_attenuate_kernel).
#include <cuda_bf16.h>

#include <algorithm>

#include "dgsm_internal.cuh"

namespace dgsm {
namespace {

constexpr int NF_FREQ = 16;
constexpr int NF_FEAT = 96;
constexpr int NF_HID = 64;
// parameter offsets (float32 master vector)
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NF_HID * NF_FEAT;
constexpr int OFF_W2 = OFF_B1 + NF_HID;
constexpr int OFF_B2 = OFF_W2 + NF_HID * NF_HID;
constexpr int OFF_W3 = OFF_B2 + NF_HID;
constexpr int OFF_B3 = OFF_W3 + NF_HID * NF_HID;
constexpr int OFF_W4 = OFF_B3 + NF_HID;
constexpr int OFF_B4 = OFF_W4 + NF_HID * NF_HID;
constexpr int OFF_W5 = OFF_B4 + NF_HID;
constexpr int OFF_B5 = OFF_W5 + NF_HID;
constexpr int NF_PARAMS = OFF_B5 + 1;  // 18753
constexpr int NF_WEIGHTS = OFF_B5;     // everything but b5 lives in shared memory

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// f_m = 2^(8m/15), m = 0..15, rounded to float32 (bit patterns, so that the
// phase f_m x is the same float32 product everywhere it is formed).
__constant__ uint32_t NF_FREQ_BITS[NF_FREQ] = {
    0x3f800000u, 0x3fb9401eu, 0x40060dbcu, 0x40420300u, 0x408c64c3u, 0x40cb2ff5u,
    0x4113088cu, 0x4154cc02u, 0x4199fcb9u, 0x41dedc67u, 0x42214518u, 0x426966a5u,
    0x42a8e5a3u, 0x42f47080u, 0x4330e285u, 0x43800000u};
__device__ __forceinline__ float nf_freq(int m) { return __uint_as_float(NF_FREQ_BITS[m]); }

// sin and cos of pi p, p = f x the float32 product, reduced exactly to
// [-1, 1] half-turns first.  The bfloat16 rounding that follows is a
// quantisation decision, so the phase is defined in float32.
__device__ __forceinline__ void nf_sincos(float f, float x, float &s, float &c) {
    float p = __fmul_rn(f, x);
    p -= 2.0f * rintf(0.5f * p);
    sincospif(p, &s, &c);
}

// Shell coordinate rho in [0, 1] of distance t for strictly increasing radii.
__device__ __forceinline__ float nf_rho(float t, const float *rs, int K) {
    const int k = count_le(rs, K, t) - 1;
    if (k < 0 || K < 2) return 0.0f;
    if (k >= K - 1) return 1.0f;
    const float w = (t - rs[k]) / (rs[k + 1] - rs[k]);
    return ((float)k + w) / (float)(K - 1);
}

// SplitMix64 (Steele, Lea, Flood 2014): one 64-bit output per counter value.
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// ---------------------------------------------------------------------------
// Training
// ---------------------------------------------------------------------------
constexpr int FB_THREADS = 128;
constexpr int ROW = NF_HID + 1;  // padded per-thread row in shared memory

// Per-sample scratch in global memory (float32): features (96), h1..h4 (4 x 64),
// dz1..dz4 (4 x 64), dy (1)  ->  NF_SAMPLE floats per sample.
constexpr int SC_H0 = 0;
constexpr int SC_H1 = SC_H0 + NF_FEAT;
constexpr int SC_DZ1 = SC_H1 + 4 * NF_HID;
constexpr int SC_DY = SC_DZ1 + 4 * NF_HID;
constexpr int NF_SAMPLE = SC_DY + 1;

// Copy the bf16-rounded weights (all but b5) into shared memory.
__device__ void nf_load_weights(const float *__restrict__ params, float *sw) {
    for (int e = threadIdx.x; e < NF_WEIGHTS; e += blockDim.x) {
        const bool is_bias = (e >= OFF_B1 && e < OFF_W2) || (e >= OFF_B2 && e < OFF_W3) ||
                             (e >= OFF_B3 && e < OFF_W4) || (e >= OFF_B4 && e < OFF_W5);
        sw[e] = is_bias ? params[e] : bf16r(params[e]);
    }
}

// One thread per sample: voxel draw (when uvr == nullptr), forward, loss,
// backward to every dz.  The thread's current input vector lives in a
// padded shared-memory row; outputs accumulate in registers.
__global__ void __launch_bounds__(FB_THREADS) nf_fwdbwd_kernel(
    const float *__restrict__ params, const float *__restrict__ atlas, int H, int W, int K,
    unsigned long long seed, const float *__restrict__ uvr_in, const float *__restrict__ tgt_in,
    int B, float *__restrict__ scratch, float *__restrict__ loss_out) {
    extern __shared__ float smem[];
    float *sw = smem;                        // NF_WEIGHTS
    float *rowbuf = sw + NF_WEIGHTS;         // FB_THREADS x ROW
    __shared__ float s_loss;
    nf_load_weights(params, sw);
    if (threadIdx.x == 0) s_loss = 0.0f;
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < B;
    float *row = rowbuf + threadIdx.x * ROW;
    float *sc = scratch + (int64_t)(live ? s : 0) * NF_SAMPLE;
    float u = 0.f, v = 0.f, rho = 0.f, target = 0.f;
    if (live) {
        if (uvr_in) {
            u = uvr_in[3 * s]; v = uvr_in[3 * s + 1]; rho = uvr_in[3 * s + 2];
            target = tgt_in[s];
        } else {
            const unsigned long long r = splitmix64(seed + (unsigned long long)s);
            const unsigned long long nvox = (unsigned long long)K * H * W;
            const unsigned long long idx = r % nvox;
            const int k = (int)(idx / ((unsigned long long)H * W));
            const int rem = (int)(idx - (unsigned long long)k * H * W);
            const int i = rem / W, j = rem - (rem / W) * W;
            u = (2.0f * j + 1.0f) / W - 1.0f;
            v = (2.0f * i + 1.0f) / H - 1.0f;
            rho = K > 1 ? (float)k / (float)(K - 1) : 0.0f;
            target = atlas[idx];
        }
    }
    float z[NF_HID];
    // ---- layer 1 from the Fourier features ----
#pragma unroll
    for (int o = 0; o < NF_HID; ++o) z[o] = sw[OFF_B1 + o];
    for (int a = 0; a < 3; ++a) {
        const float x = a == 0 ? u : (a == 1 ? v : rho);
        for (int m = 0; m < NF_FREQ; ++m) {
            float sn, cs;
            nf_sincos(nf_freq(m), x, sn, cs);
            sn = bf16r(sn);
            cs = bf16r(cs);
            if (live) {
                sc[SC_H0 + 32 * a + m] = sn;
                sc[SC_H0 + 32 * a + 16 + m] = cs;
            }
            const float *w1s = sw + OFF_W1 + 32 * a + m;
#pragma unroll
            for (int o = 0; o < NF_HID; ++o)
                z[o] = fmaf(w1s[o * NF_FEAT], sn, fmaf(w1s[o * NF_FEAT + 16], cs, z[o]));
        }
    }
    // ---- layers 2..4 ----
    for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int o = 0; o < NF_HID; ++o) {
            const float h = bf16r(fmaxf(z[o], 0.0f));
            row[o] = h;
            if (live) sc[SC_H1 + l * NF_HID + o] = h;
        }
        const float *Wl = sw + (l == 0 ? OFF_W2 : l == 1 ? OFF_W3 : OFF_W4);
        const float *bl = sw + (l == 0 ? OFF_B2 : l == 1 ? OFF_B3 : OFF_B4);
#pragma unroll
        for (int o = 0; o < NF_HID; ++o) z[o] = bl[o];
        for (int i = 0; i < NF_HID; ++i) {
            const float x = row[i];
#pragma unroll
            for (int o = 0; o < NF_HID; ++o) z[o] = fmaf(Wl[o * NF_HID + i], x, z[o]);
        }
    }
    // ---- output ----
    float y = params[OFF_B5];
#pragma unroll
    for (int o = 0; o < NF_HID; ++o) {
        const float h = bf16r(fmaxf(z[o], 0.0f));
        z[o] = h;  // z now holds h4
        if (live) sc[SC_H1 + 3 * NF_HID + o] = h;
        y = fmaf(sw[OFF_W5 + o], h, y);
    }
    const float T = 1.0f / (1.0f + expf(-y));
    const float err = live ? T - target : 0.0f;
    const float dy = 2.0f * err * T * (1.0f - T) / (float)B;
    if (live) sc[SC_DY] = dy;
    atomicAdd(&s_loss, err * err);
    // ---- backward: dz4 = dy w5 (.) [h4 > 0], then dz_{l-1} = (W_l^T dz_l) (.) [h_{l-1} > 0] ----
#pragma unroll
    for (int o = 0; o < NF_HID; ++o) {
        const float d = z[o] > 0.0f ? dy * sw[OFF_W5 + o] : 0.0f;
        row[o] = d;
        if (live) sc[SC_DZ1 + 3 * NF_HID + o] = d;
    }
    for (int l = 3; l >= 1; --l) {       // dz_l from dz_{l+1} through W_{l+1}
        const float *Wn = sw + (l == 3 ? OFF_W4 : l == 2 ? OFF_W3 : OFF_W2);
        float g[NF_HID];
#pragma unroll
        for (int i = 0; i < NF_HID; ++i) g[i] = 0.0f;
        for (int o = 0; o < NF_HID; ++o) {
            const float d = row[o];
#pragma unroll
            for (int i = 0; i < NF_HID; ++i) g[i] = fmaf(Wn[o * NF_HID + i], d, g[i]);
        }
        const float *hl = sc + SC_H1 + (l - 1) * NF_HID;
#pragma unroll
        for (int i = 0; i < NF_HID; ++i) {
            const float d = (live && hl[i] > 0.0f) ? g[i] : 0.0f;
            row[i] = d;
            if (live) sc[SC_DZ1 + (l - 1) * NF_HID + i] = d;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && loss_out) atomicAdd(loss_out, s_loss / (float)B);
}

// Weight gradients: dW_l = sum_s dz_l[s] h_{l-1}[s]^T, db_l = sum_s dz_l[s]
// (layer 5: w5, b5 from dy and h4).  Block (split, layer) reduces the samples
// of its split into partial[split][param].
constexpr int WG_THREADS = 256;
constexpr int WG_CHUNK = 32;

__global__ void __launch_bounds__(WG_THREADS) nf_wgrad_kernel(const float *__restrict__ scratch, int B,
                                                              int n_split, float *__restrict__ partial) {
    const int split = blockIdx.x, layer = blockIdx.y;  // layer 0..4
    const int n_out = layer == 4 ? 1 : NF_HID;
    const int n_in = layer == 0 ? NF_FEAT : NF_HID;
    const int in_off = layer == 0 ? SC_H0 : SC_H1 + (layer - 1) * NF_HID;
    const int dz_off = layer == 4 ? SC_DY : SC_DZ1 + layer * NF_HID;
    const int w_off = layer == 0 ? OFF_W1 : layer == 1 ? OFF_W2 : layer == 2 ? OFF_W3 : layer == 3 ? OFF_W4 : OFF_W5;
    const int b_off = layer == 0 ? OFF_B1 : layer == 1 ? OFF_B2 : layer == 2 ? OFF_B3 : layer == 3 ? OFF_B4 : OFF_B5;
    const int n_w = n_out * n_in, n_tot = n_w + n_out;
    __shared__ float sdz[WG_CHUNK][NF_HID];
    __shared__ float sh[WG_CHUNK][NF_FEAT];
    const int per = (B + n_split - 1) / n_split;
    const int s0 = split * per, s1 = min(B, s0 + per);
    constexpr int MAXO = (NF_HID * NF_FEAT + NF_HID + WG_THREADS - 1) / WG_THREADS;  // 25
    float acc[MAXO];
#pragma unroll
    for (int q = 0; q < MAXO; ++q) acc[q] = 0.0f;
    for (int c0 = s0; c0 < s1; c0 += WG_CHUNK) {
        const int cnt = min(WG_CHUNK, s1 - c0);
        for (int e = threadIdx.x; e < WG_CHUNK * NF_FEAT; e += WG_THREADS) {
            const int r = e / NF_FEAT, i = e - r * NF_FEAT;
            sh[r][i] = (r < cnt && i < n_in) ? scratch[(int64_t)(c0 + r) * NF_SAMPLE + in_off + i] : 0.0f;
        }
        for (int e = threadIdx.x; e < WG_CHUNK * NF_HID; e += WG_THREADS) {
            const int r = e / NF_HID, o = e - r * NF_HID;
            sdz[r][o] = (r < cnt && o < n_out) ? scratch[(int64_t)(c0 + r) * NF_SAMPLE + dz_off + o] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXO; ++q) {
            const int idx = threadIdx.x + q * WG_THREADS;
            if (idx >= n_tot) break;
            float a = acc[q];
            if (idx < n_w) {
                const int o = idx / n_in, i = idx - o * n_in;
                for (int r = 0; r < cnt; ++r) a = fmaf(sdz[r][o], sh[r][i], a);
            } else {
                const int o = idx - n_w;
                for (int r = 0; r < cnt; ++r) a += sdz[r][o];
            }
            acc[q] = a;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < MAXO; ++q) {
        const int idx = threadIdx.x + q * WG_THREADS;
        if (idx >= n_tot) break;
        const int p = idx < n_w ? w_off + idx : b_off + (idx - n_w);
        partial[(int64_t)split * NF_PARAMS + p] = acc[q];
    }
}

// Sum the partial gradients in split order, then Adam (or just the gradient).
__global__ void nf_adam_kernel(const float *__restrict__ partial, int n_split, float *__restrict__ params,
                               float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
                               float eps, int step, float *__restrict__ grad_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NF_PARAMS) return;
    float g = 0.0f;
    for (int s = 0; s < n_split; ++s) g += partial[(int64_t)s * NF_PARAMS + p];
    if (grad_out) {
        grad_out[p] = g;
        return;
    }
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.0f - powf(b1, (float)step));
    const float vh = vv / (1.0f - powf(b2, (float)step));
    params[p] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores
// ---------------------------------------------------------------------------
constexpr int IF_WARPS = 4;
constexpr int IF_THREADS = IF_WARPS * 32;
// shared: bf16 weights W1 (64 x 96), W2..W4 (64 x 64) in [out][in] order, then
// float biases b1..b4 (4 x 64), bf16-rounded w5 (64), b5
constexpr int IF_WB = NF_HID * NF_FEAT + 3 * NF_HID * NF_HID;   // bf16 elements
constexpr size_t IF_SMEM = IF_WB * sizeof(__nv_bfloat16) + (4 * NF_HID + NF_HID + 4) * sizeof(float);

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ void nf_stage_infer_weights(const float *__restrict__ params, __nv_bfloat16 *wb, float *fb) {
    for (int e = threadIdx.x; e < IF_WB; e += blockDim.x) {
        int src;
        if (e < NF_HID * NF_FEAT) src = OFF_W1 + e;
        else {
            const int r = e - NF_HID * NF_FEAT, l = r / (NF_HID * NF_HID), q = r - l * NF_HID * NF_HID;
            src = (l == 0 ? OFF_W2 : l == 1 ? OFF_W3 : OFF_W4) + q;
        }
        wb[e] = __float2bfloat16_rn(params[src]);
    }
    for (int e = threadIdx.x; e < 4 * NF_HID; e += blockDim.x) {
        const int l = e / NF_HID, o = e - l * NF_HID;
        fb[e] = params[(l == 0 ? OFF_B1 : l == 1 ? OFF_B2 : l == 2 ? OFF_B3 : OFF_B4) + o];
    }
    for (int e = threadIdx.x; e < NF_HID; e += blockDim.x) fb[4 * NF_HID + e] = bf16r(params[OFF_W5 + e]);
    if (threadIdx.x == 0) fb[5 * NF_HID] = params[OFF_B5];
}

// The field for 32 samples per warp (two 16-row tiles).  uvr[t][r]: the
// inputs of rows g (r = 0) and g + 8 (r = 1) of tile t, g = lane / 4.
// Returns T_hat for those four rows (valid in every lane of the row's group).
__device__ __forceinline__ void nf_field32(const __nv_bfloat16 *wb, const float *fb,
                                           const float (&uvr)[2][2][3], float (&T)[2][2]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    (void)g;
    uint32_t A[2][6][4];  // A fragments of layer 1: tile, k-tile, register
#pragma unroll
    for (int tt = 0; tt < 2; ++tt)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // this lane's frequencies m in {2t, 2t+1, 2t+8, 2t+9}
            float sn[2][4], cs[2][4];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int m = 2 * t4 + (q & 1) + (q >> 1) * 8;
                    nf_sincos(nf_freq(m), uvr[tt][r][a], sn[r][q], cs[r][q]);
                }
            // k-tile 2a holds the sines of axis a, 2a+1 its cosines
            A[tt][2 * a][0] = pack_bf16(sn[0][0], sn[0][1]);
            A[tt][2 * a][1] = pack_bf16(sn[1][0], sn[1][1]);
            A[tt][2 * a][2] = pack_bf16(sn[0][2], sn[0][3]);
            A[tt][2 * a][3] = pack_bf16(sn[1][2], sn[1][3]);
            A[tt][2 * a + 1][0] = pack_bf16(cs[0][0], cs[0][1]);
            A[tt][2 * a + 1][1] = pack_bf16(cs[1][0], cs[1][1]);
            A[tt][2 * a + 1][2] = pack_bf16(cs[0][2], cs[0][3]);
            A[tt][2 * a + 1][3] = pack_bf16(cs[1][2], cs[1][3]);
        }
    const uint32_t *wb32 = reinterpret_cast<const uint32_t *>(wb);
    uint32_t Hf[2][4][4];  // activations as A fragments (4 k-tiles of 16)
    // ---- layer 1: 96 -> 64 ----
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
        float C[8][4];
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const float b0 = fb[8 * n + 2 * t4], b1 = fb[8 * n + 2 * t4 + 1];
            C[n][0] = b0; C[n][1] = b1; C[n][2] = b0; C[n][3] = b1;
        }
#pragma unroll
        for (int kt = 0; kt < 6; ++kt)
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int o = 8 * n + (lane >> 2);
                const uint32_t b0 = wb32[(o * NF_FEAT + 16 * kt + 2 * t4) >> 1];
                const uint32_t b1 = wb32[(o * NF_FEAT + 16 * kt + 2 * t4 + 8) >> 1];
                mma_bf16(C[n], A[tt][kt][0], A[tt][kt][1], A[tt][kt][2], A[tt][kt][3], b0, b1);
            }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            Hf[tt][kt][0] = pack_bf16(fmaxf(C[2 * kt][0], 0.f), fmaxf(C[2 * kt][1], 0.f));
            Hf[tt][kt][1] = pack_bf16(fmaxf(C[2 * kt][2], 0.f), fmaxf(C[2 * kt][3], 0.f));
            Hf[tt][kt][2] = pack_bf16(fmaxf(C[2 * kt + 1][0], 0.f), fmaxf(C[2 * kt + 1][1], 0.f));
            Hf[tt][kt][3] = pack_bf16(fmaxf(C[2 * kt + 1][2], 0.f), fmaxf(C[2 * kt + 1][3], 0.f));
        }
    }
    // ---- layers 2..4: 64 -> 64 ----
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const uint32_t *Wl = wb32 + ((NF_HID * NF_FEAT + l * NF_HID * NF_HID) >> 1);
        const float *bl = fb + (l + 1) * NF_HID;
#pragma unroll
        for (int tt = 0; tt < 2; ++tt) {
            float C[8][4];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const float b0 = bl[8 * n + 2 * t4], b1 = bl[8 * n + 2 * t4 + 1];
                C[n][0] = b0; C[n][1] = b1; C[n][2] = b0; C[n][3] = b1;
            }
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    const int o = 8 * n + (lane >> 2);
                    const uint32_t b0 = Wl[(o * NF_HID + 16 * kt + 2 * t4) >> 1];
                    const uint32_t b1 = Wl[(o * NF_HID + 16 * kt + 2 * t4 + 8) >> 1];
                    mma_bf16(C[n], Hf[tt][kt][0], Hf[tt][kt][1], Hf[tt][kt][2], Hf[tt][kt][3], b0, b1);
                }
            if (l < 2) {
#pragma unroll
                for (int kt = 0; kt < 4; ++kt) {
                    Hf[tt][kt][0] = pack_bf16(fmaxf(C[2 * kt][0], 0.f), fmaxf(C[2 * kt][1], 0.f));
                    Hf[tt][kt][1] = pack_bf16(fmaxf(C[2 * kt][2], 0.f), fmaxf(C[2 * kt][3], 0.f));
                    Hf[tt][kt][2] = pack_bf16(fmaxf(C[2 * kt + 1][0], 0.f), fmaxf(C[2 * kt + 1][1], 0.f));
                    Hf[tt][kt][3] = pack_bf16(fmaxf(C[2 * kt + 1][2], 0.f), fmaxf(C[2 * kt + 1][3], 0.f));
                }
            } else {
                // output layer: y = w5 . bf16(ReLU(z4)) + b5, reduced over the 4 lanes of a row group
                const float *w5 = fb + 4 * NF_HID;
                float y0 = 0.f, y1 = 0.f;
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    const int c = 8 * n + 2 * t4;
                    y0 = fmaf(w5[c], bf16r(fmaxf(C[n][0], 0.f)), y0);
                    y0 = fmaf(w5[c + 1], bf16r(fmaxf(C[n][1], 0.f)), y0);
                    y1 = fmaf(w5[c], bf16r(fmaxf(C[n][2], 0.f)), y1);
                    y1 = fmaf(w5[c + 1], bf16r(fmaxf(C[n][3], 0.f)), y1);
                }
                y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
                y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
                y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
                y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
                const float b5 = fb[5 * NF_HID];
                T[tt][0] = 1.0f / (1.0f + expf(-(y0 + b5)));
                T[tt][1] = 1.0f / (1.0f + expf(-(y1 + b5)));
            }
        }
    }
}

// Field values at n explicit inputs (u, v, rho).
__global__ void __launch_bounds__(IF_THREADS) nf_infer_kernel(const float *__restrict__ params,
                                                              const float *__restrict__ uvr, int64_t n,
                                                              float *__restrict__ T_out) {
    extern __shared__ float4 smem_if[];
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(smem_if);
    float *fb = reinterpret_cast<float *>(wb + IF_WB);
    nf_stage_infer_weights(params, wb, fb);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
    for (int64_t base = ((int64_t)blockIdx.x * IF_WARPS + warp) * 32; base < n;
         base += (int64_t)gridDim.x * IF_WARPS * 32) {
        float in[2][2][3], T[2][2];
#pragma unroll
        for (int tt = 0; tt < 2; ++tt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int64_t s = base + 16 * tt + g + 8 * r;
#pragma unroll
                for (int a = 0; a < 3; ++a) in[tt][r][a] = s < n ? uvr[3 * s + a] : 0.f;
            }
        nf_field32(wb, fb, in, T);
        if ((lane & 3) == 0)
#pragma unroll
            for (int tt = 0; tt < 2; ++tt)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int64_t s = base + 16 * tt + g + 8 * r;
                    if (s < n) T_out[s] = T[tt][r];
                }
    }
}

// Per-tile worst error of the field against the exact atlas over all voxels
// of the tile (tile x tile texels x K shells): one block per tile.
__global__ void __launch_bounds__(IF_THREADS) nf_tile_error_kernel(
    const float *__restrict__ params, const float *__restrict__ atlas, int H, int W, int K, int tile,
    int tx, float *__restrict__ tile_err) {
    extern __shared__ float4 smem_if[];
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(smem_if);
    float *fb = reinterpret_cast<float *>(wb + IF_WB);
    __shared__ float s_err;
    nf_stage_infer_weights(params, wb, fb);
    if (threadIdx.x == 0) s_err = 0.0f;
    __syncthreads();
    const int t = blockIdx.x, ti = t / tx, tj = t - ti * tx;
    const int i0 = ti * tile, j0 = tj * tile;
    const int hh = min(tile, H - i0), ww = min(tile, W - j0);
    const int nvox = hh * ww * K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
    float worst = 0.0f;
    for (int base = warp * 32; base < nvox; base += IF_WARPS * 32) {
        float in[2][2][3], T[2][2], ref[2][2];
#pragma unroll
        for (int tt = 0; tt < 2; ++tt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                int e = base + 16 * tt + g + 8 * r;
                const bool ok = e < nvox;
                e = ok ? e : 0;
                const int k = e / (hh * ww), rem = e - k * hh * ww;
                const int i = i0 + rem / ww, j = j0 + rem % ww;
                in[tt][r][0] = (2.0f * j + 1.0f) / W - 1.0f;
                in[tt][r][1] = (2.0f * i + 1.0f) / H - 1.0f;
                in[tt][r][2] = K > 1 ? (float)k / (float)(K - 1) : 0.0f;
                ref[tt][r] = ok ? atlas[((int64_t)k * H + i) * W + j] : -1.0f;
            }
        nf_field32(wb, fb, in, T);
#pragma unroll
        for (int tt = 0; tt < 2; ++tt)
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (ref[tt][r] >= 0.0f) worst = fmaxf(worst, fabsf(T[tt][r] - ref[tt][r]));
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) atomicMax(reinterpret_cast<int *>(&s_err), __float_as_int(worst));
    __syncthreads();
    if (threadIdx.x == 0) tile_err[t] = s_err;
}

// Attenuation through the field: per query and light the field value at
// (u, v, rho) of the query, or -- where the light's fallback mask marks the
// tile of the query's texel cell -- the exact trilinear atlas lookup.  The
// weights of up to NF_LGROUP lights are staged in shared memory once per
// block; with more lights, launches over light groups carry the weighted sum
// in `accum` (first group writes it, last group turns it into colours).
constexpr int NF_LGROUP = 4;
constexpr int NA_WARPS = 8;   // one block per SM: 8 warps share the staged weights
constexpr int NA_THREADS = NA_WARPS * 32;

__global__ void __launch_bounds__(NA_THREADS, 1) nf_attenuate_kernel(
    const float *__restrict__ params, int n_params_stride, const uint8_t *__restrict__ mask,
    const float *__restrict__ atlas, int L, int l0, int LG, int H, int W,
    const float *__restrict__ radii, int K, int tile, int tx, int n_tiles,
    const float *__restrict__ lights, const float *__restrict__ qm, const float *cin, int64_t Q,
    const float *__restrict__ lw, float wd, float *cout, float *__restrict__ Tout,
    float *__restrict__ accum) {
    extern __shared__ float4 smem_if[];
    __shared__ float rs[256];
    __shared__ float ls[64 * 3];
    __shared__ float wl[64];
    for (int k = threadIdx.x; k < K; k += blockDim.x) rs[k] = radii[k];
    for (int k = threadIdx.x; k < 3 * L; k += blockDim.x) ls[k] = lights[k];
    for (int k = threadIdx.x; k < L; k += blockDim.x) wl[k] = lw ? lw[k] : 1.0f / (float)L;
    char *stage_base = reinterpret_cast<char *>(smem_if);
    for (int lg = 0; lg < LG; ++lg) {
        __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(stage_base + lg * IF_SMEM);
        nf_stage_infer_weights(params + (int64_t)(l0 + lg) * n_params_stride, wb,
                               reinterpret_cast<float *>(wb + IF_WB));
    }
    __syncthreads();
    const bool first = l0 == 0, last = l0 + LG == L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
    const int64_t plane = (int64_t)H * W;
    for (int64_t base = ((int64_t)blockIdx.x * NA_WARPS + warp) * 32; base < Q;
         base += (int64_t)gridDim.x * NA_WARPS * 32) {
        float px[2][2], py[2][2], pz[2][2], acc[2][2];
#pragma unroll
        for (int tt = 0; tt < 2; ++tt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int64_t s = base + 16 * tt + g + 8 * r;
                const bool ok = s < Q;
                px[tt][r] = ok ? qm[3 * s] : 0.f;
                py[tt][r] = ok ? qm[3 * s + 1] : 0.f;
                pz[tt][r] = ok ? qm[3 * s + 2] : 0.f;
                acc[tt][r] = (ok && !first) ? accum[s] : 0.f;
            }
        for (int lg = 0; lg < LG; ++lg) {
            const int l = l0 + lg;
            const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(stage_base + lg * IF_SMEM);
            const float *fb = reinterpret_cast<const float *>(wb + IF_WB);
            float in[2][2][3], T[2][2];
            SampleIndex si[2][2];
#pragma unroll
            for (int tt = 0; tt < 2; ++tt)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    si[tt][r] = sample_index(px[tt][r], py[tt][r], pz[tt][r], ls[3 * l], ls[3 * l + 1],
                                             ls[3 * l + 2], H, W, rs, K);
                    const float2 uv = xencode(px[tt][r] - ls[3 * l], py[tt][r] - ls[3 * l + 1],
                                              pz[tt][r] - ls[3 * l + 2]);
                    in[tt][r][0] = uv.x;
                    in[tt][r][1] = uv.y;
                    in[tt][r][2] = nf_rho(si[tt][r].t, rs, K);
                }
            nf_field32(wb, fb, in, T);
#pragma unroll
            for (int tt = 0; tt < 2; ++tt)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const SampleIndex &sx = si[tt][r];
                    float Tl = T[tt][r];
                    if (sx.t == 0.0f) Tl = 1.0f;
                    else if (mask && mask[(int64_t)l * n_tiles + (sx.ci / tile) * tx + (sx.cj / tile)]) {
                        // exact trilinear lookup in the fallback atlas
                        const int j0 = min(max(sx.bj, 0), W - 1), j1 = min(max(sx.bj + 1, 0), W - 1);
                        const int i0 = min(max(sx.bi, 0), H - 1), i1 = min(max(sx.bi + 1, 0), H - 1);
                        int k0, k1;
                        float wt;
                        if (sx.k < 0) { k0 = k1 = 0; wt = 0.f; }
                        else if (sx.k >= K - 1) { k0 = k1 = K - 1; wt = 0.f; }
                        else { k0 = sx.k; k1 = sx.k + 1; wt = (sx.t - rs[k0]) / (rs[k1] - rs[k0]); }
                        const float *A0 = atlas + (int64_t)l * K * plane + k0 * plane;
                        const float *A1 = atlas + (int64_t)l * K * plane + k1 * plane;
                        const float fx = sx.fx, fy = sx.fy;
                        const float b0 = (1 - fy) * ((1 - fx) * A0[i0 * W + j0] + fx * A0[i0 * W + j1]) +
                                         fy * ((1 - fx) * A0[i1 * W + j0] + fx * A0[i1 * W + j1]);
                        const float b1 = (1 - fy) * ((1 - fx) * A1[i0 * W + j0] + fx * A1[i0 * W + j1]) +
                                         fy * ((1 - fx) * A1[i1 * W + j0] + fx * A1[i1 * W + j1]);
                        Tl = (1 - wt) * b0 + wt * b1;
                    }
                    const int64_t q = base + 16 * tt + g + 8 * r;
                    if (Tout && q < Q && (lane & 3) == 0) Tout[q * L + l] = Tl;
                    acc[tt][r] = fmaf(wl[l], Tl, acc[tt][r]);
                }
        }
        if ((lane & 3) == 0)
#pragma unroll
            for (int tt = 0; tt < 2; ++tt)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int64_t q = base + 16 * tt + g + 8 * r;
                    if (q >= Q) continue;
                    if (!last) {
                        accum[q] = acc[tt][r];
                        continue;
                    }
                    const float f = 1.0f - wd + wd * acc[tt][r];
                    const float c0 = cin[3 * q], c1 = cin[3 * q + 1], c2 = cin[3 * q + 2];
                    cout[3 * q] = c0 * f;
                    cout[3 * q + 1] = c1 * f;
                    cout[3 * q + 2] = c2 * f;
                }
    }
}

// He-uniform initial weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)), zero biases.
__global__ void nf_init_kernel(unsigned long long seed, float *__restrict__ params) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NF_PARAMS) return;
    int fan_in = 0;
    if (p < OFF_B1) fan_in = NF_FEAT;
    else if ((p >= OFF_W2 && p < OFF_B2) || (p >= OFF_W3 && p < OFF_B3) || (p >= OFF_W4 && p < OFF_B4) ||
             (p >= OFF_W5 && p < OFF_B5))
        fan_in = NF_HID;
    if (fan_in == 0) {
        params[p] = 0.0f;
        return;
    }
    const unsigned long long r = splitmix64(seed * (unsigned long long)NF_PARAMS + (unsigned long long)p);
    const float u01 = (float)(r >> 40) * (1.0f / 16777216.0f);  // 24 random bits
    params[p] = (2.0f * u01 - 1.0f) * sqrtf(6.0f / (float)fan_in);
}

int set_infer_smem(dgsm_ctx *ctx) {
    cudaError_t e = cudaFuncSetAttribute(nf_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)IF_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nf_tile_error_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)IF_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nf_attenuate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(NF_LGROUP * IF_SMEM));
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf: smem attribute");
}

// scratch: per-sample rows + partial gradients of n_split splits
int nf_scratch(dgsm_ctx *ctx, int B, int n_split, float **rows, float **partial) {
    void *p;
    const size_t bytes = sizeof(float) * ((size_t)B * NF_SAMPLE + (size_t)n_split * NF_PARAMS);
    int rc = ws_reserve(ctx, WS_NF, bytes, &p);
    if (rc) return rc;
    *rows = (float *)p;
    *partial = *rows + (size_t)B * NF_SAMPLE;
    return DGSM_OK;
}

constexpr size_t FB_SMEM = (size_t)(NF_WEIGHTS + FB_THREADS * ROW) * sizeof(float);

int run_fwdbwd(dgsm_ctx *ctx, const float *params, const float *atlas, int H, int W, int K,
               unsigned long long seed, const float *uvr, const float *tgt, int B, int n_split,
               float *rows, float *partial, float *loss_slot, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(nf_fwdbwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FB_SMEM);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nf: smem attribute");
    nf_fwdbwd_kernel<<<(B + FB_THREADS - 1) / FB_THREADS, FB_THREADS, FB_SMEM, s>>>(
        params, atlas, H, W, K, seed, uvr, tgt, B, rows, loss_slot);
    nf_wgrad_kernel<<<dim3(n_split, 5), WG_THREADS, 0, s>>>(rows, B, n_split, partial);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf forward/backward");
}

}  // namespace
}  // namespace dgsm

using namespace dgsm;

extern "C" int64_t nf_param_count(void) { return NF_PARAMS; }

extern "C" int nf_init(dgsm_ctx *ctx, uint64_t seed, float *params, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!params) return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_init: null params");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    nf_init_kernel<<<(NF_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, params);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf_init_kernel");
}

extern "C" int nf_loss_grad(dgsm_ctx *ctx, const float *params, const float *uvr, const float *target,
                            int64_t n, float *loss_out, float *grad_out, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 1 || n > (1 << 24) || !params || !uvr || !target || !grad_out)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_loss_grad: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int B = (int)n, n_split = std::max(1, std::min(64, B / 64));
    float *rows, *partial;
    int rc = nf_scratch(ctx, B, n_split, &rows, &partial);
    if (rc) return rc;
    if (loss_out && (e = cudaMemsetAsync(loss_out, 0, sizeof(float), s)) != cudaSuccess)
        return cuda_fail(ctx, e, "nf: memset");
    if ((rc = run_fwdbwd(ctx, params, nullptr, 1, 1, 1, 0ull, uvr, target, B, n_split, rows, partial,
                         loss_out, s)))
        return rc;
    nf_adam_kernel<<<(NF_PARAMS + 255) / 256, 256, 0, s>>>(partial, n_split, nullptr, nullptr, nullptr,
                                                           0.f, 0.f, 0.f, 0.f, 1, grad_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf_loss_grad");
}

extern "C" int nf_train(dgsm_ctx *ctx, const float *atlas, int32_t H, int32_t W, int32_t K,
                        float *params, float *adam_m, float *adam_v, int32_t steps, int32_t batch,
                        float lr, uint64_t seed, int32_t step0, float *loss_out, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!atlas || !params || !adam_m || !adam_v || H < 1 || W < 1 || K < 1 || steps < 0 || batch < 1 ||
        batch > (1 << 22) || step0 < 0 || !(lr > 0.f))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_train: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int n_split = std::max(1, std::min(128, batch / 64));
    float *rows, *partial;
    int rc = nf_scratch(ctx, batch, n_split, &rows, &partial);
    if (rc) return rc;
    if (loss_out && steps > 0 && (e = cudaMemsetAsync(loss_out, 0, sizeof(float) * steps, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "nf: memset");
    for (int it = 0; it < steps; ++it) {
        const int step = step0 + it + 1;
        const unsigned long long sd = splitmix64(seed ^ (0x51ED270B3A1C5Full * (unsigned long long)step));
        if ((rc = run_fwdbwd(ctx, params, atlas, H, W, K, sd, nullptr, nullptr, batch, n_split, rows, partial,
                             loss_out ? loss_out + it : nullptr, s)))
            return rc;
        nf_adam_kernel<<<(NF_PARAMS + 255) / 256, 256, 0, s>>>(partial, n_split, params, adam_m, adam_v, lr,
                                                               0.9f, 0.999f, 1e-8f, step, nullptr);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf_train");
}

extern "C" int nf_forward(dgsm_ctx *ctx, const float *params, const float *uvr, int64_t n, float *T_out,
                          void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!params || !uvr || !T_out))) return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_forward: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n == 0) return DGSM_OK;
    int rc = set_infer_smem(ctx);
    if (rc) return rc;
    const int grid = (int)std::min<int64_t>((n + IF_THREADS - 1) / IF_THREADS, (int64_t)ctx->num_sms * 8);
    nf_infer_kernel<<<grid, IF_THREADS, IF_SMEM, (cudaStream_t)stream>>>(params, uvr, n, T_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf_infer_kernel");
}

extern "C" int nf_tile_error(dgsm_ctx *ctx, const float *params, const float *atlas, int32_t H, int32_t W,
                             int32_t K, int32_t tile, float *tile_err, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!params || !atlas || !tile_err || H < 1 || W < 1 || K < 1 || tile < 1)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_tile_error: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    int rc = set_infer_smem(ctx);
    if (rc) return rc;
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    nf_tile_error_kernel<<<tx * ty, IF_THREADS, IF_SMEM, (cudaStream_t)stream>>>(params, atlas, H, W, K, tile,
                                                                                tx, tile_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf_tile_error_kernel");
}

extern "C" int nf_attenuate(dgsm_ctx *ctx, const float *params, const uint8_t *mask, const float *atlas,
                            int32_t L, int32_t H, int32_t W, const float *radii, int32_t K, int32_t tile,
                            const float *lights, const float *q_means, const float *colors_in, int64_t n_q,
                            const float *light_w, float direct_frac, float *colors_out, float *T_out,
                            void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n_q < 0 || L < 1 || L > 64 || H < 1 || W < 1 || H > 4096 || W > 4096 || K < 1 || K > 256 || tile < 1 ||
        !params || !radii || !lights || (mask && !atlas))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_attenuate: bad arguments");
    if (n_q > 0 && (!q_means || !colors_in || !colors_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_attenuate: null query array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n_q == 0) return DGSM_OK;
    int rc = set_infer_smem(ctx);
    if (rc) return rc;
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    const int grid = (int)std::min<int64_t>((n_q + NA_THREADS - 1) / NA_THREADS, (int64_t)ctx->num_sms);
    float *accum = nullptr;
    if (L > NF_LGROUP) {
        void *p;
        if ((rc = ws_reserve(ctx, WS_NF_ACC, sizeof(float) * (size_t)n_q, &p))) return rc;
        accum = (float *)p;
    }
    for (int l0 = 0; l0 < L; l0 += NF_LGROUP) {
        const int LG = std::min(NF_LGROUP, L - l0);
        nf_attenuate_kernel<<<grid, NA_THREADS, LG * IF_SMEM, (cudaStream_t)stream>>>(
            params, NF_PARAMS, mask, atlas, L, l0, LG, H, W, radii, K, tile, tx, tx * ty, lights, q_means,
            colors_in, n_q, light_w, direct_frac, colors_out, T_out, accum);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf_attenuate_kernel");
}
