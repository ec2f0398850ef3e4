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
// Inference: 5th-generation tensor cores (tcgen05.mma kind::f16, bf16
// operands in shared memory, FP32 accumulators in tensor memory), 128 rows
// per warpgroup tile (tc::field_kernel); attenuation writes T per light and a
// small pass forms the colours (tc::combine_kernel).
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
// bf16 packing for the tensor-core operands
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
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

// ---------------------------------------------------------------------------
// Inference on the 5th-generation tensor cores (tcgen05).
//
// One warpgroup (128 threads) per CTA; thread t owns row t of a 128-row tile
// (one query, voxel or input).  Per layer, the row's inputs (bf16) are written
// to shared memory in the no-swizzle K-major canonical layout (8-row x 16-byte
// core matrices; element (r, k) at (r/8) SBO + (k/8) 128 + (r%8) 16 + (k%8) 2),
// one thread issues the MMAs (M = 128, N = 64, K = 16 each; kind::f16, bf16 in,
// f32 out) into a 64-column TMEM accumulator and commits them to an mbarrier,
// and every thread reads its row back with tcgen05.ld for the bias, ReLU and
// bf16 rounding of the next layer's input.  The weights of the CTA's light
// stay in shared memory in the same layout (B operands: W[out][in], K-major).
// ---------------------------------------------------------------------------
namespace tc {

constexpr int TM = 128;
constexpr int WG = 2;                 // warpgroups per CTA, each with its own tile in flight
constexpr int THREADS = 128 * WG;
// K of each layer: inputs, then two constant-1 columns that carry the bias as
// a bfloat16 hi + lo pair (exact to ~2^-18 relative), padded to 16
constexpr int K1 = NF_FEAT + 16;      // 112
constexpr int KH = NF_HID + 16;       // 80
constexpr int N5 = 16;                // output layer: column 0 = w5, the rest zero
constexpr uint32_t SBO1 = (K1 / 8) * 128;   // 1792
constexpr uint32_t SBOH = (KH / 8) * 128;   // 1280
constexpr uint32_t W1_BYTES = NF_HID * K1 * 2;   // 14336
constexpr uint32_t WL_BYTES = NF_HID * KH * 2;   // 10240
constexpr uint32_t W5_BYTES = N5 * KH * 2;       // 2560
constexpr uint32_t A_BYTES = TM * K1 * 2;        // 28672 (also holds the K = 80 layout)
constexpr uint32_t OFF_SW1 = 0;
constexpr uint32_t OFF_SW2 = OFF_SW1 + W1_BYTES;
constexpr uint32_t OFF_SW5 = OFF_SW2 + 3 * WL_BYTES;
constexpr uint32_t OFF_SA = OFF_SW5 + W5_BYTES;       // one A tile per warpgroup
constexpr uint32_t OFF_BAR = OFF_SA + WG * A_BYTES;   // one mbarrier per warpgroup
constexpr uint32_t SMEM = OFF_BAR + 8 * WG + 128;     // + alignment slack
// instruction descriptors: f32 accumulate, bf16 A and B, both K-major, M = 128
constexpr uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
constexpr long long WAIT_LIMIT = 1ll << 24;

__device__ __forceinline__ uint32_t canon(int r, int k, uint32_t sbo) {
    return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for phase `parity` of the mbarrier: at most `limit` polls;
// false on timeout.
__device__ __forceinline__ bool bar_wait_n(uint32_t bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) { return bar_wait_n(bar, parity, WAIT_LIMIT); }

// Self-test of the bounded wait: one mbarrier expecting one arrival.  With
// `arrive` the thread arrives first and the wait completes; without, nothing
// arrives, the wait gives up after `limit` polls, and the kernel records
// DGSM_ERR_TIMEOUT in the status word and returns normally.
__global__ void wait_selftest_kernel(int arrive, long long limit, int *status) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) bar_init(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
        if (!bar_wait_n(b, 0u, limit)) record_status(status, DGSM_ERR_TIMEOUT);
    }
}

// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// one fp32 column of this thread's TMEM lane
__device__ __forceinline__ float ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

// bf16 pair (lo in the low half) of ReLU(lo), ReLU(hi)
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void st_bf16(char *sm, uint32_t off, float x) {
    *reinterpret_cast<__nv_bfloat16 *>(sm + off) = __float2bfloat16_rn(x);
}

// Stage one light's weights as bf16 B operands (rows = outputs, K-major):
// [W_l | b_hi b_lo 0 ...] for the four hidden layers and [w5 | b5_hi b5_lo 0 ...]
// as row 0 of the 16-row output operand.
__device__ void stage_weights(const float *__restrict__ params, char *sm) {
    for (int e = threadIdx.x; e < NF_HID * K1; e += blockDim.x) {
        const int n = e / K1, k = e - n * K1;
        const float b = params[OFF_B1 + n], bh = bf16r(b);
        const float v = k < NF_FEAT ? params[OFF_W1 + n * NF_FEAT + k] : k == NF_FEAT ? bh : k == NF_FEAT + 1 ? b - bh : 0.f;
        st_bf16(sm, OFF_SW1 + canon(n, k, SBO1), v);
    }
    for (int e = threadIdx.x; e < 3 * NF_HID * KH; e += blockDim.x) {
        const int l = e / (NF_HID * KH), q = e - l * NF_HID * KH, n = q / KH, k = q - n * KH;
        const int w = l == 0 ? OFF_W2 : l == 1 ? OFF_W3 : OFF_W4, bo = l == 0 ? OFF_B2 : l == 1 ? OFF_B3 : OFF_B4;
        const float b = params[bo + n], bh = bf16r(b);
        const float v = k < NF_HID ? params[w + n * NF_HID + k] : k == NF_HID ? bh : k == NF_HID + 1 ? b - bh : 0.f;
        st_bf16(sm, OFF_SW2 + l * WL_BYTES + canon(n, k, SBOH), v);
    }
    for (int e = threadIdx.x; e < N5 * KH; e += blockDim.x) {
        const int n = e / KH, k = e - n * KH;
        const float b = params[OFF_B5], bh = bf16r(b);
        const float v = n != 0 ? 0.f : k < NF_HID ? params[OFF_W5 + k] : k == NF_HID ? bh : k == NF_HID + 1 ? b - bh : 0.f;
        st_bf16(sm, OFF_SW5 + canon(n, k, SBOH), v);
    }
}

// sin and cos of pi p for the float32 phase p = f x reduced exactly to
// [-1, 1] half-turns, by the SFU (absolute error ~1e-6, far below the
// bfloat16 spacing the feature is rounded to next).
__device__ __forceinline__ void sincos_sfu(float f, float x, float &s, float &c) {
    float p = __fmul_rn(f, x);
    p -= 2.0f * rintf(0.5f * p);
    const float a = p * 3.14159265358979f;
    s = __sinf(a);
    c = __cosf(a);
}

// the constant columns (1, 1, 0, ..., 0) at k0 .. k0 + 15 of row r
__device__ __forceinline__ void write_ones(char *sA, int r, int k0, uint32_t sbo) {
    const uint32_t one2 = 0x3F803F80u;  // two bf16 ones
    *reinterpret_cast<uint4 *>(sA + canon(r, k0, sbo)) = make_uint4(one2 & 0xFFFFFFFFu, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(sA + canon(r, k0 + 8, sbo)) = make_uint4(0u, 0u, 0u, 0u);
}

// The 96 bf16 features of (u, v, rho) as row r of the layer-1 A tile:
// k = 32 axis + m (sin), 32 axis + 16 + m (cos); 8 features per 16-byte store;
// then the two bias columns.
__device__ __forceinline__ void write_features(char *sA, int r, float u, float v, float rho) {
    const float x[3] = {u, v, rho};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // frequencies 8h .. 8h+7
            float sn[8], cs[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) sincos_sfu(nf_freq(8 * h + m), x[a], sn[m], cs[m]);
            uint4 ws, wc;
            ws.x = pack_bf16(sn[0], sn[1]); ws.y = pack_bf16(sn[2], sn[3]);
            ws.z = pack_bf16(sn[4], sn[5]); ws.w = pack_bf16(sn[6], sn[7]);
            wc.x = pack_bf16(cs[0], cs[1]); wc.y = pack_bf16(cs[2], cs[3]);
            wc.z = pack_bf16(cs[4], cs[5]); wc.w = pack_bf16(cs[6], cs[7]);
            *reinterpret_cast<uint4 *>(sA + canon(r, 32 * a + 8 * h, SBO1)) = ws;
            *reinterpret_cast<uint4 *>(sA + canon(r, 32 * a + 16 + 8 * h, SBO1)) = wc;
        }
    }
    write_ones(sA, r, NF_FEAT, SBO1);
}

// Issue one layer's MMAs and commit them to the barrier.
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t a_saddr, uint32_t b_saddr, int kdim, int n,
                                            uint32_t bar) {
    const uint32_t sbo = (uint32_t)(kdim / 8) * 128u, id = idesc(n);
    for (int s = 0; s < kdim / 16; ++s)
        mma(tmem, sdesc(a_saddr + 256u * s, 128u, sbo), sdesc(b_saddr + 256u * s, 128u, sbo), id, s > 0 ? 1u : 0u);
    commit(bar);
}

// Hidden-layer epilogue of row r: h = bf16(ReLU(z)) (the bias is in z) into
// the A tile in the K = 80 layout; after layer 1 also its bias columns.
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, char *sA, int r, bool first) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float z[32];
        ld32(trow + 32u * half, z);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint4 w;
            w.x = relu_bf16x2(z[8 * g + 0], z[8 * g + 1]);
            w.y = relu_bf16x2(z[8 * g + 2], z[8 * g + 3]);
            w.z = relu_bf16x2(z[8 * g + 4], z[8 * g + 5]);
            w.w = relu_bf16x2(z[8 * g + 6], z[8 * g + 7]);
            *reinterpret_cast<uint4 *>(sA + canon(r, 32 * half + 8 * g, SBOH)) = w;
        }
    }
    if (first) write_ones(sA, r, NF_HID, SBOH);
}

// The field for the warpgroup's current tile: its A tile already holds the
// features.  r = row (thread within the warpgroup).  Returns false if an
// MMA completion wait timed out.
__device__ __forceinline__ void wg_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

__device__ __forceinline__ bool run_mlp(uint32_t sbase, char *sA, int g, int r, uint32_t tmem, uint32_t &phase,
                                        float &T) {
    const int warp = r >> 5;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t a_saddr = sbase + OFF_SA + (uint32_t)g * A_BYTES, bar = sbase + OFF_BAR + 8u * g;
    bool ok = true;
    for (int layer = 0; layer < 5; ++layer) {
        fence_async_smem();
        fence_before();
        wg_sync(g);
        if (r == 0) {
            fence_after();
            if (layer == 0) issue_layer(tmem, a_saddr, sbase + OFF_SW1, K1, NF_HID, bar);
            else if (layer < 4) issue_layer(tmem, a_saddr, sbase + OFF_SW2 + (layer - 1) * WL_BYTES, KH, NF_HID, bar);
            else issue_layer(tmem, a_saddr, sbase + OFF_SW5, KH, N5, bar);
        }
        ok = bar_wait(bar, phase) && ok;
        phase ^= 1u;
        fence_after();
        if (layer < 4) hidden_epilogue(trow, sA, r, layer == 0);
        else T = 1.0f / (1.0f + expf(-ld1(trow)));
    }
    fence_before();
    wg_sync(g);  // TMEM and A are free for the next tile
    return ok;
}

enum Mode { MODE_UVR = 0, MODE_VOXEL_ERR = 1, MODE_QUERY = 2 };

// MODE_UVR: T_out[i] = field(uvr[i]) for i < n.
// MODE_VOXEL_ERR: one atlas tile per work unit, tile_err[t] = max |field - atlas|
//   over its tile x tile texels x K shells.
// MODE_QUERY: light l = blockIdx.x % L; per query q, T_all[l Q + q] = the
//   field at (u, v, rho) of q seen from light l, or the exact trilinear atlas
//   lookup where mask[l][tile of q's texel cell] is set.
template <int MODE>
__global__ void __launch_bounds__(THREADS, 2) field_kernel(
    const float *__restrict__ params, int n_params_stride, int64_t n, const float *__restrict__ uvr,
    const float *__restrict__ atlas, int H, int W, int K, int tile, int tx, int n_tiles,
    const float *__restrict__ radii, const float *__restrict__ lights, int L, const uint8_t *__restrict__ mask,
    float *__restrict__ out, int *__restrict__ status) {
    extern __shared__ __align__(1024) char smem_raw[];
    char *sm = reinterpret_cast<char *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
    __shared__ uint32_t s_tmem;
    __shared__ float rs[256];
    __shared__ float s_err[WG];
    const int tid = threadIdx.x, warp = tid >> 5, g = tid >> 7, r = tid & 127;
    const int l = MODE == MODE_QUERY ? (int)(blockIdx.x % (unsigned)L) : 0;
    // work units (tiles of 128 rows) are dealt to warpgroups
    const int cta = MODE == MODE_QUERY ? (int)(blockIdx.x / (unsigned)L) : (int)blockIdx.x;
    const int n_cta = MODE == MODE_QUERY ? (int)(gridDim.x / (unsigned)L) : (int)gridDim.x;
    const int wgi = cta * WG + g, n_wg = n_cta * WG;
    stage_weights(params + (int64_t)l * n_params_stride, sm);
    if (MODE == MODE_QUERY)
        for (int k = tid; k < K; k += blockDim.x) rs[k] = radii[k];
    if (tid < WG) bar_init(sbase + OFF_BAR + 8u * tid);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(64u * WG)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem + 64u * g;   // this warpgroup's 64 columns
    uint32_t phase = 0;
    bool ok = true;
    char *sA = sm + OFF_SA + (uint32_t)g * A_BYTES;
    if (MODE == MODE_UVR || MODE == MODE_QUERY) {
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (MODE == MODE_QUERY) { ox = lights[3 * l]; oy = lights[3 * l + 1]; oz = lights[3 * l + 2]; }
        // the next tile's inputs are loaded while this tile runs its MMA chain
        const int64_t step = (int64_t)n_wg * TM;
        float nx = 0.f, ny = 0.f, nz = 0.f;
        {
            const int64_t q0 = (int64_t)wgi * TM + r;
            if (q0 < n) { nx = uvr[3 * q0]; ny = uvr[3 * q0 + 1]; nz = uvr[3 * q0 + 2]; }
        }
        for (int64_t base = (int64_t)wgi * TM; base < n; base += step) {
            const int64_t q = base + r;
            const bool valid = q < n;
            const float ix = nx, iy = ny, iz = nz;
            if (q + step < n) { nx = uvr[3 * (q + step)]; ny = uvr[3 * (q + step) + 1]; nz = uvr[3 * (q + step) + 2]; }
            float u = 0.f, v = 0.f, rho = 0.f;
            SampleIndex si;
            si.t = 0.f;
            if (valid) {
                if (MODE == MODE_UVR) {
                    u = ix; v = iy; rho = iz;
                } else {
                    si = sample_index(ix, iy, iz, ox, oy, oz, H, W, rs, K);
                    const float2 e = xencode(ix - ox, iy - oy, iz - oz);
                    u = e.x; v = e.y;
                    rho = nf_rho(si.t, rs, K);
                }
            }
            write_features(sA, r, u, v, rho);
            float T = 0.f;
            ok = run_mlp(sbase, sA, g, r, tmem, phase, T) && ok;
            if (!valid) continue;
            if (MODE == MODE_UVR) {
                out[q] = T;
            } else {
                if (si.t == 0.0f) T = 1.0f;
                else if (mask && mask[(int64_t)l * n_tiles + (si.ci / tile) * tx + (si.cj / tile)]) {
                    const int j0 = min(max(si.bj, 0), W - 1), j1 = min(max(si.bj + 1, 0), W - 1);
                    const int i0 = min(max(si.bi, 0), H - 1), i1 = min(max(si.bi + 1, 0), H - 1);
                    int k0, k1;
                    float wt;
                    if (si.k < 0) { k0 = k1 = 0; wt = 0.f; }
                    else if (si.k >= K - 1) { k0 = k1 = K - 1; wt = 0.f; }
                    else { k0 = si.k; k1 = si.k + 1; wt = (si.t - rs[k0]) / (rs[k1] - rs[k0]); }
                    const int64_t plane = (int64_t)H * W;
                    const float *A0 = atlas + (int64_t)l * K * plane + k0 * plane;
                    const float *A1 = atlas + (int64_t)l * K * plane + k1 * plane;
                    const float fx = si.fx, fy = si.fy;
                    const float b0 = (1 - fy) * ((1 - fx) * A0[i0 * W + j0] + fx * A0[i0 * W + j1]) +
                                     fy * ((1 - fx) * A0[i1 * W + j0] + fx * A0[i1 * W + j1]);
                    const float b1 = (1 - fy) * ((1 - fx) * A1[i0 * W + j0] + fx * A1[i0 * W + j1]) +
                                     fy * ((1 - fx) * A1[i1 * W + j0] + fx * A1[i1 * W + j1]);
                    T = (1 - wt) * b0 + wt * b1;
                }
                out[(int64_t)l * n + q] = T;
            }
        }
    } else {
        // atlas tiles as work units of a warpgroup; a tile's voxels in rows of 128
        for (int t = wgi; t < n_tiles; t += n_wg) {
            const int ti = t / tx, tj = t - ti * tx;
            const int i0 = ti * tile, j0 = tj * tile;
            const int hh = min(tile, H - i0), ww = min(tile, W - j0);
            const int nvox = hh * ww * K;
            float worst = 0.f;
            for (int vb = 0; vb < nvox; vb += TM) {
                const int e = vb + r;
                const bool valid = e < nvox;
                const int ee = valid ? e : 0;
                const int k = ee / (hh * ww), rem = ee - k * hh * ww;
                const int i = i0 + rem / ww, j = j0 + rem % ww;
                const float u = (2.0f * j + 1.0f) / W - 1.0f, v = (2.0f * i + 1.0f) / H - 1.0f;
                const float rho = K > 1 ? (float)k / (float)(K - 1) : 0.0f;
                write_features(sA, r, u, v, rho);
                float T = 0.f;
                ok = run_mlp(sbase, sA, g, r, tmem, phase, T) && ok;
                if (valid) worst = fmaxf(worst, fabsf(T - atlas[((int64_t)k * H + i) * W + j]));
            }
            for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
            if (r == 0) s_err[g] = 0.f;
            wg_sync(g);
            if ((r & 31) == 0) atomicMax(reinterpret_cast<int *>(&s_err[g]), __float_as_int(worst));
            wg_sync(g);
            if (r == 0) out[t] = s_err[g];
        }
    }
    if (!ok && tid == 0) record_status(status, DGSM_ERR_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(64u * WG)
                     : "memory");
    }
}

template <int MODE>
int launch_field(dgsm_ctx *ctx, int grid, cudaStream_t s, const float *params, int stride, int64_t n,
                 const float *uvr, const float *atlas, int H, int W, int K, int tile, int tx, int n_tiles,
                 const float *radii, const float *lights, int L, const uint8_t *mask, float *out) {
    cudaError_t e = cudaFuncSetAttribute(field_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nf: tcgen05 smem attribute");
    field_kernel<MODE><<<grid, THREADS, SMEM, s>>>(params, stride, n, uvr, atlas, H, W, K, tile, tx, n_tiles,
                                                    radii, lights, L, mask, out, ctx->d_status);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf: tcgen05 field kernel");
}

// c' = c (1 - wd + wd sum_l w_l T_all[l][q]); optional T_out[q][l].
__global__ void combine_kernel(const float *__restrict__ T_all, int L, int64_t Q, const float *__restrict__ lw,
                               float wd, const float *cin, float *cout, float *__restrict__ Tout) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int l = 0; l < L; ++l) {
            const float T = T_all[(int64_t)l * Q + q];
            if (Tout) Tout[q * L + l] = T;
            acc = fmaf(lw ? lw[l] : 1.0f / (float)L, T, acc);
        }
        const float f = 1.0f - wd + wd * acc;
        const float c0 = cin[3 * q], c1 = cin[3 * q + 1], c2 = cin[3 * q + 2];
        cout[3 * q] = c0 * f;
        cout[3 * q + 1] = c1 * f;
        cout[3 * q + 2] = c2 * f;
    }
}

}  // namespace tc

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
    DGSM_RANGE("nf_train");
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
    if (n < 0 || !params || (n > 0 && (!uvr || !T_out))) return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_forward: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n == 0) return DGSM_OK;
    const int per_cta = tc::TM * tc::WG;
    const int grid = (int)std::min<int64_t>((n + per_cta - 1) / per_cta, (int64_t)ctx->num_sms * 2);
    return tc::launch_field<tc::MODE_UVR>(ctx, grid, (cudaStream_t)stream, params, NF_PARAMS, n, uvr, nullptr, 0, 0,
                                          0, 1, 1, 0, nullptr, nullptr, 1, nullptr, T_out);
}

extern "C" int nf_tile_error(dgsm_ctx *ctx, const float *params, const float *atlas, int32_t H, int32_t W,
                             int32_t K, int32_t tile, float *tile_err, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (!params || !atlas || !tile_err || H < 1 || W < 1 || K < 1 || tile < 1)
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_tile_error: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    const int grid = std::max(1, std::min((tx * ty + tc::WG - 1) / tc::WG, ctx->num_sms * 2));
    return tc::launch_field<tc::MODE_VOXEL_ERR>(ctx, grid, (cudaStream_t)stream, params, NF_PARAMS, 0, nullptr, atlas,
                                                H, W, K, tile, tx, tx * ty, nullptr, nullptr, 1, nullptr, tile_err);
}

extern "C" int nf_attenuate(dgsm_ctx *ctx, const float *params, const uint8_t *mask, const float *atlas,
                            int32_t L, int32_t H, int32_t W, const float *radii, int32_t K, int32_t tile,
                            const float *lights, const float *q_means, const float *colors_in, int64_t n_q,
                            const float *light_w, float direct_frac, float *colors_out, float *T_out,
                            void *stream) {
    DGSM_RANGE("nf_attenuate");
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (n_q < 0 || L < 1 || L > 64 || H < 1 || W < 1 || H > 4096 || W > 4096 || K < 1 || K > 256 || tile < 1 ||
        !params || !radii || !lights || (mask && !atlas))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_attenuate: bad arguments");
    if (n_q > 0 && (!q_means || !colors_in || !colors_out))
        return fail(ctx, DGSM_ERR_INVALID_ARG, "nf_attenuate: null query array");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (n_q == 0) return DGSM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    void *p;
    int rc = ws_reserve(ctx, WS_NF_ACC, sizeof(float) * (size_t)L * n_q, &p);
    if (rc) return rc;
    float *T_all = (float *)p;
    const int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    // CTAs per light: enough for two per SM in all, no more than the light's tiles of rows
    const int64_t rows_per_cta = tc::TM * tc::WG;
    const int per_light = (int)std::max<int64_t>(
        1, std::min<int64_t>((n_q + rows_per_cta - 1) / rows_per_cta, std::max(1, 2 * ctx->num_sms / L)));
    rc = tc::launch_field<tc::MODE_QUERY>(ctx, per_light * L, s, params, NF_PARAMS, n_q, q_means, atlas, H, W, K,
                                          tile, tx, tx * ty, radii, lights, L, mask, T_all);
    if (rc) return rc;
    const int cgrid = (int)std::min<int64_t>((n_q + 255) / 256, (int64_t)ctx->num_sms * 8);
    tc::combine_kernel<<<cgrid, 256, 0, s>>>(T_all, L, n_q, light_w, direct_frac, colors_in, colors_out, T_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "nf: combine kernel");
}

extern "C" int dgsm_selftest_wait(dgsm_ctx *ctx, int32_t arrive, int64_t limit, void *stream) {
    if (!ctx) return DGSM_ERR_INVALID_ARG;
    if (limit < 1 || limit > (1ll << 24)) return fail(ctx, DGSM_ERR_INVALID_ARG, "selftest: limit in 1..2^24");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    tc::wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(arrive, (long long)limit, ctx->d_status);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGSM_OK : cuda_fail(ctx, e, "wait_selftest_kernel");
}
