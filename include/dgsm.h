/*
 * dgsm.h -- C ABI of libdgsm.so: Deep Gaussian Shadow Maps on one B300
 * (sm_103a).  Method: "Animated 3DGS Avatars in Diverse Scenes with
 * Consistent Lighting and Shadows", Sec. 3.2 (build), 3.3 (sampling),
 * 3.4 (HDRI probe fit) and 3.5 (radiance transfer).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Array pointers are DEVICE pointers into caller-owned memory unless an
 *   argument says "host".  Arrays are dense, C-contiguous, float32 unless
 *   stated; the library never keeps them past the call and never frees them.
 * - Gaussians come as structure-of-arrays: means (n,3) metres; scales (n,3)
 *   linear standard deviations (not log), all > 0; quats (n,4) rotations
 *   (w,x,y,z), normalised inside; opac (n) opacities alpha, clamped to
 *   [0, 1-1e-6].  Covariance Sigma = R diag(s^2) R^T, precision A = Sigma^-1.
 * - An atlas is [L][K][H][W] (lights, shells, rows, columns) of
 *   transmittance T (Eq. 4); row i holds v_i = (2i+1)/H - 1, column j holds
 *   u_j = (2j+1)/W - 1 of the octahedral map (Eq. 6); shell k holds T at
 *   distance radii[k] from the light.  radii must be strictly increasing
 *   and > 0.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *   enqueued asynchronously unless the function says it blocks.
 * - Return value: DGSM_OK (0) or one of the dgsm_status codes; details
 *   via dgsm_last_error(ctx).  Nothing traps or aborts on bad input.
 * - A dgsm_ctx is bound to one device and must not be used by two host
 *   threads at once.
 */
#ifndef DGSM_H
#define DGSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgsm_ctx dgsm_ctx;
typedef struct dgsm_graph dgsm_graph;

enum dgsm_status {
    DGSM_OK = 0,
    DGSM_ERR_INVALID_ARG = 1,      /* a size, pointer or parameter is out of range */
    DGSM_ERR_CUDA = 2,             /* a CUDA runtime call failed (message names it) */
    DGSM_ERR_WORKSPACE = 3,        /* an output or internal capacity is too small */
    DGSM_ERR_TIMEOUT = 4,          /* a bounded device-side wait gave up */
    DGSM_ERR_NONFINITE_INPUT = 5,  /* NaN/Inf or non-positive scale in the Gaussians */
    DGSM_ERR_NOT_SPD = 6           /* the SH normal equations are not positive definite */
};

enum dgsm_dtype { DGSM_F32 = 0, DGSM_F16 = 1, DGSM_BF16 = 2 };

/* Build parameters.  kappa: global strength knob of Eq. 5 (default 1).
 * eps_cull: optical depth a culled Gaussian may still carry along a ray
 * (default 1e-7); it sets each Gaussian's culling radius k (Mahalanobis
 * units), k^2 = 2 ln2 * max(e,1), e the binary exponent of
 * kappa * alpha/(1-alpha) * (s_max/s_min) / eps_cull.
 * tile: atlas tile edge in texels for light-space binning: 8 or 16 for
 * dgsm_build (default 8, the paper's 8x8 tiles), also 4 for dgsm_bin.
 * chunk: Gaussians staged in shared memory per round, 16..192 (default 128);
 * a tile's list is processed in work items of at most 8 chunks.
 * atlas_dtype: storage type of T (dgsm_dtype; tau is always accumulated in
 * float32).
 * max_pairs: 0 (default) sizes the pair buffers from the exact pair counts,
 * read back twice during the build; > 0 sizes them for max_pairs pairs
 * (both the (super-tile, Gaussian) and the (tile, Gaussian) pairs; see
 * dgsm_build_stats) and never blocks (so the build can be captured in a CUDA graph; see
 * dgsm_graph_begin).  A build whose pairs exceed max_pairs records
 * DGSM_ERR_WORKSPACE in the status word and leaves T = 1 in its atlas.
 * beta_mode: the opacity-to-absorption mapping (ablation (B) of Sec. 4),
 * with tau* = -ln(1 - alpha):
 *   1: beta = kappa tau*;
 *   2: beta = kappa tau* sqrt(tr(A)/3) / sqrt(2 pi), A the precision (Eq. 5,
 *      the default);
 *   3: beta = kappa tau* / ((2 pi)^(3/2) sqrt(det Sigma)), Sigma the covariance;
 *   4: beta = kappa tau* / ((2 pi)^(3/2) s_x s_y s_z); for Sigma = R diag(s^2) R^T
 *      sqrt(det Sigma) = s_x s_y s_z, so 4 computes the same value as 3.
 * The culling radius keeps the eps_cull bound under every mapping: the
 * factor (s_max/s_min) above becomes sqrt(2 pi) s_max (mapping 1) or
 * s_max / (2 pi s_x s_y s_z) (mappings 3, 4).
 * atlas_map: the atlas parameterisation (ablation (C) of Sec. 4): 0 the
 * octahedral map of Eq. 6 (the default); 1 a cube map of six F x F faces
 * stacked in rows (H = 6F, W = F, F a multiple of the tile): face f holds
 * rows [f F, (f+1) F) and its texel (u, v) looks along F_f + u U_f + v V_f
 * with the cube-map axes (F, U, V) = (+x, -z, -y), (-x, +z, -y), (+y, +x, +z),
 * (-y, +x, -z), (+z, +x, -y), (-z, -x, -y).  Cube atlases are read with
 * dgsm_attenuate_cube. */
typedef struct {
    float kappa;
    float eps_cull;
    int32_t tile;
    int32_t chunk;
    int32_t atlas_dtype;
    int32_t max_pairs;
    int32_t beta_mode;
    int32_t atlas_map;
} dgsm_params;

/* Receiver-driven region of interest of dgsm_build_roi (device pointers). */
typedef struct {
    const float *recv_means; /* (n_recv,3) receiver centres, for instance the scene Gaussians */
    int64_t n_recv;
    const float *box;        /* 5 floats c_x, c_y, R, z_min, z_max (dgsm_roi_box writes them) */
    uint8_t *mask_out;       /* (n_lights,H,W) or NULL: 1 on the texels of P, else 0 */
    int32_t *krange_out;     /* (n_lights,2) or NULL: k_min, k_max (k_max = -1: empty) */
} dgsm_roi;

/* Counters of the last dgsm_build on a context. */
typedef struct {
    int64_t n_pairs;      /* binned (tile, Gaussian) pairs */
    int64_t rays_tested;  /* texel-ray x Gaussian pairs tested (texels x list lengths) */
    int64_t ray_evals;    /* Gaussian-ray evaluations: rays cutting the culling ellipsoid at t > 0 */
    int64_t shell_evals;  /* closed-form (Eq. 3) evaluations at shell radii */
    int64_t n_super_pairs; /* binned (8x8-tile super-tile, Gaussian) pairs */
} dgsm_build_stats;

/* Transfer parameters of Eqs. 9-10: lobe exponent q (1 = Lambertian),
 * global intensity gamma, clip t_max, epsilon of the denominator, and the
 * lat-long grid n_theta x n_phi (cell centres, weights sin(theta)).
 * Defaults: q=1, gamma=1, t_max=10, eps=1e-8, 32 x 64. */
typedef struct {
    float q;
    float gamma;
    float t_max;
    float eps;
    int32_t n_theta;
    int32_t n_phi;
} dgsm_relight_params;

void dgsm_default_params(dgsm_params *p);
void dgsm_default_relight_params(dgsm_relight_params *p);

/* Create a context on `device` (makes it current).  The context owns a
 * growable device workspace used by dgsm_build; it is freed by
 * dgsm_destroy.  Returns DGSM_OK or DGSM_ERR_CUDA. */
int dgsm_create(int device, dgsm_ctx **out);
void dgsm_destroy(dgsm_ctx *ctx);

/* Message of the last failure on ctx (static storage of the context;
 * valid until the next call on it). */
const char *dgsm_last_error(const dgsm_ctx *ctx);
const char *dgsm_status_string(int status);

/* Deep Gaussian Shadow Map build (Sec. 3.2, Eqs. 1-5; tile binning after
 * the occluder-culling paragraph).  For every light l, texel (i,j) and
 * shell k:  atlas[l][k][i][j] = exp(-sum_n beta_n I_n(d_ij, radii[k])),
 * beta_n from Eq. 5, I_n the closed form of Eq. 3 along the ray from
 * lights[l] through the decoded texel centre d_ij.  Gaussians whose
 * culling ellipsoid does not reach a tile (or a shell interval) are
 * skipped; each skip changes tau by at most params->eps_cull.
 *   means/scales/quats/opac: the n occluder Gaussians (n >= 0; n = 0 gives
 *   T = 1 everywhere); lights: (n_lights,3), 1 <= n_lights <= 64;
 *   1 <= H, W <= 4096; radii: (K), 1 <= K <= 256; params: host pointer or
 *   NULL for defaults; atlas: [n_lights][K][H][W] of params->atlas_dtype.
 * With params->max_pairs = 0 it blocks twice to size the workspace from the
 * numbers of binned pairs; with max_pairs > 0 it never blocks and
 * reports input errors through the status word (dgsm_sync_status): a
 * non-finite Gaussian is then left out of the atlas.  Within a voxel the
 * contributions of different Gaussians are summed in an order that can vary
 * from run to run (float32 atomics), so repeated builds agree to rounding,
 * not bit for bit.  Fails with
 * DGSM_ERR_NONFINITE_INPUT if an input Gaussian has a NaN/Inf field or a
 * scale <= 0, DGSM_ERR_WORKSPACE if more than 2^31 pairs are binned, and
 * DGSM_ERR_INVALID_ARG for max_pairs = 0 on a stream that is capturing. */
int dgsm_build(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
               const float *opac, int64_t n, const float *lights, int32_t n_lights, int32_t H,
               int32_t W, const float *radii, int32_t K, const dgsm_params *params, void *atlas,
               void *stream);

/* dgsm_build restricted to a receiver-driven region of interest (Sec. 3.2,
 * "Receiver-driven ROI"; the timing ablation (D) of Sec. 4).  Receivers
 * whose centres lie in the box B = {|x - c_x| <= R, |y - c_y| <= R,
 * z_min <= z <= z_max} are projected into each light's atlas; P is the set
 * of texels their trilinear lookups read (the 2 x 2 bilinear taps of each,
 * clamped to the edge) and [k_min, k_max] the shells that bracket their
 * distances.  On R = P x {k_min..k_max} the atlas equals dgsm_build's; on
 * every other voxel it is 1.  Only tiles holding a texel of P are binned and
 * evaluated, and Gaussians wholly beyond shell k_max are skipped, so the
 * cost follows the region, not the atlas.  Receivers in B are attenuated by
 * dgsm_attenuate exactly as with the dense atlas (up to summation order).
 * The box test and the projections use the single-precision index decisions
 * of dgsm_sample_index.  Other arguments, blocking and errors as for
 * dgsm_build; roi: host pointer (its arrays are device pointers). */
int dgsm_build_roi(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                   const float *opac, int64_t n, const float *lights, int32_t n_lights, int32_t H,
                   int32_t W, const float *radii, int32_t K, const dgsm_params *params,
                   const dgsm_roi *roi, void *atlas, void *stream);

/* One band of atlas rows, for splitting one light's atlas over several GPUs
 * (each GPU bins every Gaussian but builds only the tiles of its rows, then
 * the bands are exchanged; the lights themselves are independent problems).
 * Builds rows [row0, row1) of the atlas exactly as dgsm_build does and sets
 * every other texel to T = 1 (a region of interest made of whole rows).
 * 0 <= row0 < row1 <= H; other arguments, blocking and errors as for
 * dgsm_build. */
int dgsm_build_band(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                    const float *opac, int64_t n, const float *lights, int32_t n_lights, int32_t H,
                    int32_t W, const float *radii, int32_t K, const dgsm_params *params, int32_t row0,
                    int32_t row1, void *atlas, void *stream);

/* Copies `rows` rows of every plane between two row-major stacks of planes
 * of width W: dst plane p, rows [dst_row0, dst_row0 + rows) <- src plane p,
 * rows [src_row0, src_row0 + rows); planes of src_rows and dst_rows rows.
 * Cuts an atlas band out of an atlas [L][K][H][W] (planes = L K) into a
 * slab, and puts a gathered slab back.  src, dst: device; elem_bytes 4
 * (float32) or 2 (float16, bfloat16).  One asynchronous 2-D copy. */
int dgsm_atlas_rows_copy(dgsm_ctx *ctx, const void *src, int32_t src_rows, int32_t src_row0, void *dst,
                         int32_t dst_rows, int32_t dst_row0, int32_t rows, int64_t planes, int32_t W,
                         int32_t elem_bytes, void *stream);

/* The box of a region of interest around an avatar (Sec. 3.2): c = the
 * alpha-weighted centroid of the avatar's Gaussians (x, y), the given
 * half-width R, and z from the lowest to the highest avatar centre padded by
 * z_margin.  avatar_means (n,3), avatar_opac (n): device, n >= 1; box_out:
 * device, 5 floats (c_x, c_y, R, z_min, z_max; R = -1, an empty box, if the
 * opacities sum to 0).  Asynchronous; one block. */
int dgsm_roi_box(dgsm_ctx *ctx, const float *avatar_means, const float *avatar_opac, int64_t n,
                 float R, float z_margin, float *box_out, void *stream);

/* Counters of the last dgsm_build on ctx (blocks until they are ready). */
int dgsm_get_build_stats(dgsm_ctx *ctx, dgsm_build_stats *out);

/* The light-space tile binning of dgsm_build on its own (Sec. 3.2, the
 * occluder-culling paragraph: tiles are binned by the Gaussian's projected
 * footprint).  A Gaussian enters a tile's list when its bounding-sphere cone
 * overlaps the tile's (and its 8x8 super-tile's) direction cone and its
 * culling ellipsoid reaches the tile's polyhedral cone (no edge plane of the
 * tile separates it); the test of the plane between the tile's halves gives a
 * 2-bit mask of the halves (rows [0, tile/2) and [tile/2, tile)) its rays can
 * hit.  All decisions are IEEE single-precision operations in a fixed order.
 * Writes the sorted pairs key = l * n_tiles + tile (tiles row-major,
 * ceil(H/tile) x ceil(W/tile) per light), value = Gaussian index | mask << 30
 * (bit 30 top half, bit 31 bottom half), ordered by (key, Gaussian index).
 * keys_out/vals_out: device arrays of `capacity` uint32 (may be NULL when
 * capacity is 0); *n_pairs_out (host) receives the pair count.  Returns
 * DGSM_ERR_WORKSPACE (after setting *n_pairs_out) when capacity is short.
 * n < 2^30.  Blocks. */
int dgsm_bin(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
             const float *opac, int64_t n, const float *lights, int32_t n_lights, int32_t H,
             int32_t W, const float *radii, int32_t K, const dgsm_params *params,
             uint32_t *keys_out, uint32_t *vals_out, int64_t capacity, int64_t *n_pairs_out,
             void *stream);

/* Receiver attenuation (Sec. 3.3, centre sample): for each query q and
 * light l, T_l = trilinear lookup of atlas[l] at the octahedral code of
 * (x_q - o_l) and distance t = |x_q - o_l| -- bilinear between texel
 * centres with clamp-to-edge, linear between the shells bracketing t
 * (clamped to the first/last shell), T = 1 when x_q = o_l; multiplied by
 * the same lookup in atlas_dyn when it is not NULL.  Then
 *   colors_out[q] = colors_in[q] * (1 - direct_frac + direct_frac * sum_l w_l T_l)
 * with w_l = light_w[l], or 1/n_lights when light_w is NULL.
 *   atlas, atlas_dyn: [n_lights][K][H][W] of `dtype` (both the same shape);
 *   q_means, colors_in, colors_out: (n_q,3) (colors_out may equal
 *   colors_in); T_out: (n_q, n_lights) or NULL.  n_q >= 0. */
int dgsm_attenuate(dgsm_ctx *ctx, const void *atlas, const void *atlas_dyn, int32_t dtype,
                   int32_t n_lights, int32_t H, int32_t W, const float *radii, int32_t K,
                   const float *lights, const float *q_means, const float *colors_in,
                   int64_t n_q, const float *light_w, float direct_frac, float *colors_out,
                   float *T_out, void *stream);

/* dgsm_attenuate with a dynamic atlas of its own resolution and shells
 * (for instance per-frame avatar occluders at 256x256x32 beside a static
 * scene at 512x512x64): T_l = T_static,l(x) * T_dyn,l(x), each atlas
 * sampled at its own octahedral index and shell bracket.  atlas:
 * [n_lights][K][H][W], atlas_dyn: [n_lights][K_dyn][H_dyn][W_dyn], both of
 * `dtype`; radii_dyn: device, K_dyn floats.  Other arguments and errors as
 * for dgsm_attenuate. */
int dgsm_attenuate_dyn(dgsm_ctx *ctx, const void *atlas, int32_t dtype, int32_t n_lights,
                       int32_t H, int32_t W, const float *radii, int32_t K, const void *atlas_dyn,
                       int32_t H_dyn, int32_t W_dyn, const float *radii_dyn, int32_t K_dyn,
                       const float *lights, const float *q_means, const float *colors_in,
                       int64_t n_q, const float *light_w, float direct_frac, float *colors_out,
                       float *T_out, void *stream);

/* Footprint sampling for dgsm_attenuate (Sec. 3.3, last paragraph; Sec. 4,
 * ablation (A)).  The paper averages several atlas lookups over each
 * receiver's footprint instead of one lookup at its centre, with
 * rotation-aware offsets in the receiver's principal axes:
 *   x_i = mu + R (s (.) z_i),   T_l = sum_i w_i T_l(x_i),   sum_i w_i = 1,
 * then scales the colour as dgsm_attenuate does.
 *   mode DGSM_FP_CENTRE: z = 0 (the same result as dgsm_attenuate);
 *   mode DGSM_FP_STENCIL7: z in {0, +-e_x, +-e_y, +-e_z}, weights proportional
 *     to exp(-|z|^2/2) (1 at the centre, e^-1/2 on the axes);
 *   mode DGSM_FP_MC (the paper's default): n_samples offsets z ~ N(0, I),
 *     w = 1/n_samples.  Normal j of receiver q (coordinate j % 3 of sample
 *     j / 3) comes from Philox4x64-10 (Salmon et al., SC 2011) at counter
 *     (q, j / 8, 0, 0) and key (seed, 0): word (j % 8) / 2 gives two 24-bit
 *     uniforms u1, u2 in (0, 1] (top bits of its low and high halves) and
 *     Box-Muller gives sqrt(-2 ln u1) cos(2 pi u2) (even j) or sin (odd j).
 *   q_quats (n_q,4) w,x,y,z; q_scales (n_q,3) linear standard deviations;
 *   n_samples in 1..32 (DGSM_FP_MC only).  Other arguments as for
 *   dgsm_attenuate (one atlas; no dynamic atlas).  Returns DGSM_OK,
 *   DGSM_ERR_INVALID_ARG or DGSM_ERR_CUDA. */
enum dgsm_footprint { DGSM_FP_CENTRE = 0, DGSM_FP_STENCIL7 = 1, DGSM_FP_MC = 2 };
int dgsm_attenuate_footprint(dgsm_ctx *ctx, const void *atlas, int32_t dtype, int32_t n_lights,
                             int32_t H, int32_t W, const float *radii, int32_t K,
                             const float *lights, const float *q_means, const float *q_quats,
                             const float *q_scales, const float *colors_in, int64_t n_q,
                             const float *light_w, float direct_frac, int32_t mode,
                             int32_t n_samples, uint64_t seed, float *colors_out, float *T_out,
                             void *stream);

/* dgsm_attenuate on a cube-map atlas (dgsm_params.atlas_map = 1): atlas
 * [n_lights][K][6F][F] of `dtype`.  The point's face is that of the largest
 * component of x - o (ties go to x, then y; a component >= 0 picks the
 * positive face), u = U.v / m and v = V.v / m with m that component's size;
 * the bilinear taps are clamped to the face's F x F texels (no filtering
 * across faces), and shells as for dgsm_attenuate.  One atlas (no dynamic
 * atlas).  Other arguments and errors as for dgsm_attenuate. */
int dgsm_attenuate_cube(dgsm_ctx *ctx, const void *atlas, int32_t dtype, int32_t n_lights, int32_t F,
                        const float *radii, int32_t K, const float *lights, const float *q_means,
                        const float *colors_in, int64_t n_q, const float *light_w, float direct_frac,
                        float *colors_out, float *T_out, void *stream);

/* The integer decisions of dgsm_attenuate_cube, as dgsm_sample_index gives
 * them for the octahedral map: rows are global (face f's rows start at f F). */
int dgsm_sample_index_cube(dgsm_ctx *ctx, const float *points, int64_t n, const float *light, int32_t F,
                           const float *radii, int32_t K, int32_t *idx_out, float *frac_out, void *stream);

/* The integer decisions of dgsm_attenuate for n points seen from one light
 * (device pointer to 3 floats): idx_out (n,5) = texel cell row i, cell
 * column j, bilinear base row i0, base column j0, shell k (#{radii <= t}-1,
 * -1 below radii[0]); frac_out (n,3) = fy, fx, t.  Uses the same device code
 * as dgsm_attenuate. */
int dgsm_sample_index(dgsm_ctx *ctx, const float *points, int64_t n, const float *light,
                      int32_t H, int32_t W, const float *radii, int32_t K, int32_t *idx_out,
                      float *frac_out, void *stream);

/* HDRI probe fit (Sec. 3.4, Eq. 7): the weighted ridge least squares
 * (B^T W B + lambda I) A = B^T W Y over n cubemap samples, B the real SH
 * basis to degree 2 (index l^2+l+m, no Condon-Shortley phase), solved in
 * FP64 on the GPU (accumulation and Cholesky).
 *   dirs (n,3) unit directions, rgb (n,3) radiance, w (n) solid-angle
 *   weights; n >= 1; lambda >= 0.  sh_out: (3,9) float32, SH[c][k] = A[k][c];
 *   sh64_out: (3,9) float64 or NULL.  A system that is not positive
 *   definite is reported through dgsm_sync_status as DGSM_ERR_NOT_SPD and
 *   leaves sh_out zero. */
int sh_fit(dgsm_ctx *ctx, const float *dirs, const float *rgb, const float *w, int64_t n,
           double lambda, float *sh_out, double *sh64_out, void *stream);

/* 3DGS splatting into pinhole cameras: the final composite of the relit
 * avatar in the shadowed scene (Fig. 2's last stage), and the engine of
 * dgsm_render_cubemap.  Camera c is 16 floats: a rotation R (row-major; rows
 * the image x axis, the image y axis and the forward axis, world to view),
 * the position, fx, fy, cx, cy; pixel (i, j) (row i, column j, centre at
 * (j + 0.5, i + 0.5)) sees the view point (x, y, z) at (fx x/z + cx,
 * fy y/z + cy).  Splatting follows 3DGS: the screen covariance is the
 * Jacobian of this projection at the Gaussian's mean (its x/z, y/z clamped to
 * 1.3 x the half field of view) applied to the view-space covariance, plus
 * 0.3 pixel^2; a Gaussian contributes to the pixels whose centres lie within
 * Mahalanobis distance 3 of its projected mean, with alpha = min(0.99,
 * opacity exp(-m^2/2)); all of them are composited front to back by view
 * depth (ties by Gaussian index), C += alpha T c, T *= 1 - alpha, except what
 * lies behind a transmittance below 1e-6 (less than 1e-6 of the brightest
 * colour); the background is black.  Gaussians whose depth is not above
 * `near` are left out.  The inclusion test and the depth order are
 * IEEE single-precision operations in a fixed order.
 *   means, scales, quats, opac, colors: the n Gaussians (device);
 *   cams: device, n_views x 16 floats, 1 <= n_views <= 64; 1 <= W, H <= 4096;
 *   near > 0; rgb_out: device (n_views, H, W, 3); n_pairs_out: host, the
 *   (8x8 tile, splat) pairs rendered, or NULL.
 * Blocks once to size its buffers from the pair count.  Returns DGSM_OK,
 * DGSM_ERR_INVALID_ARG, DGSM_ERR_WORKSPACE or DGSM_ERR_CUDA. */
int dgsm_render_views(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                      const float *opac, const float *colors, int64_t n, const float *cams, int32_t n_views,
                      int32_t W, int32_t H, float near, float *rgb_out, int64_t *n_pairs_out, void *stream);

/* The cubemap probe of Sec. 3.4: the 3DGS scene rendered on the six
 * 90-degree cube faces at `centre` (for instance the avatar's alpha-weighted
 * centroid from dgsm_weighted_centroid), face x face pixels each.  Pixel (i, j)
 * of face f looks along F_f + u_j U_f + v_i V_f with u_j = (2j+1)/face - 1,
 * v_i = (2i+1)/face - 1 and the cube-map axes (F, U, V) = (+x, -z, -y),
 * (-x, +z, -y), (+y, +x, +z), (-y, +x, -z), (+z, +x, -y), (-z, -x, -y)
 * (dgsm_cube_dirs gives the same directions).  Each face is a
 * dgsm_render_views camera at `centre` with rows (U, V, F) and
 * fx = fy = cx = cy = face / 2 (a 90-degree field of view); splatting and
 * compositing as there.
 *   means, scales, quats, opac, colors: the n scene Gaussians (device);
 *   centre: device, 3 floats; face: a multiple of 8 in 8..1024; near > 0;
 *   rgb_out: device (6 * face * face, 3), faces in the order above, rows i,
 *   columns j; n_pairs_out: host, the (tile, splat) pairs rendered, or NULL.
 * Blocks once to size its buffers from the pair count.  Returns DGSM_OK,
 * DGSM_ERR_INVALID_ARG, DGSM_ERR_WORKSPACE or DGSM_ERR_CUDA. */
int dgsm_render_cubemap(dgsm_ctx *ctx, const float *means, const float *scales, const float *quats,
                        const float *opac, const float *colors, int64_t n, const float *centre,
                        int32_t face, float near, float *rgb_out, int64_t *n_pairs_out, void *stream);

/* Directions and solid angles of the probe's pixels (Sec. 3.4: the
 * per-pixel solid-angle weights that correct the cube map's area
 * distortion): dirs_out (6 * face * face, 3) unit texel-centre directions in
 * dgsm_render_cubemap's order, w_out (6 * face * face) the exact solid angle
 * of each texel (sum 4 pi), computed in double precision.  Device pointers;
 * asynchronous. */
int dgsm_cube_dirs(dgsm_ctx *ctx, int32_t face, float *dirs_out, float *w_out, void *stream);

/* Self-test of the library's bounded device-side waits (failure detection;
 * the paper has no counterpart).  Every wait on an mbarrier (the tensor-core
 * kernels of the surrogate) polls a bounded number of times, then records
 * DGSM_ERR_TIMEOUT in the context's status word and lets the kernel return,
 * so that the context stays usable.  This entry point runs one such wait on
 * an mbarrier that expects one arrival: with arrive != 0 the arrival comes
 * and the wait completes; with arrive = 0 nothing arrives and the wait gives
 * up after `limit` polls (1..2^24).  Read the outcome with dgsm_sync_status.
 * Returns DGSM_OK, DGSM_ERR_INVALID_ARG or DGSM_ERR_CUDA. */
int dgsm_selftest_wait(dgsm_ctx *ctx, int32_t arrive, int64_t limit, void *stream);

/* sh_fit without a context and without allocating device memory.  The paper
 * has no counterpart: this exists for callers that cannot call cudaMalloc --
 * a real-time frame loop in which cudaMalloc/cudaFree would synchronise the
 * device and stall the frame, or a host that owns all device memory through
 * its own pool.  The same computation as sh_fit (FP64 normal equations and
 * Cholesky on the current device); its per-block partial sums live in a
 * fixed array compiled into the library (147,712 bytes, held on every device
 * that loads the library until the process exits).
 *   dirs, rgb, w, n, lambda, sh_out, sh64_out: as for sh_fit, device pointers;
 *   n <= 4,194,304 (larger n returns DGSM_ERR_WORKSPACE);
 *   status_out: device int or NULL; receives DGSM_OK or DGSM_ERR_NOT_SPD
 *   (then sh_out is zero).
 * The first call on a device looks up the array's device address and keeps
 * it with the id of the context it was taken in; a call whose current
 * context differs (after cudaDeviceReset, for instance) looks it up again.
 * Make the first call, and the first after a reset, before any stream
 * capture.
 * An error that earlier work left pending on the calling thread is returned
 * as DGSM_ERR_CUDA without being cleared.  All calls share the one array:
 * calls that overlap on the GPU (on concurrent streams) race and give wrong
 * results; serialise them.  Returns DGSM_OK, DGSM_ERR_INVALID_ARG,
 * DGSM_ERR_WORKSPACE (n too large) or DGSM_ERR_CUDA; there is no context to
 * hold a message. */
int sh_fit_static(const float *dirs, const float *rgb, const float *w, int64_t n, double lambda,
                  float *sh_out, double *sh64_out, int *status_out, void *stream);

/* Per-Gaussian radiance transfer (Sec. 3.5, Eqs. 8-10):
 *   s_c(n) = clip_[0,t_max]( sum_j w_j L_c(w_j) S_j / (sum_j w_j S_j + eps) ),
 *   S_j = max(0, <w_j, n>)^q,  colors_out = max(0, gamma * colors_in (.) s).
 * n is normals[g] (normalised) when normals is not NULL, else the
 * smallest-scale axis of the Gaussian (first on ties) turned to point away
 * from `centroid` (device pointer, 3 floats).  sh: (3,9) device float32.
 * colors_out may equal colors_in.  params: host pointer or NULL. */
int sh_relight(dgsm_ctx *ctx, const float *sh, const float *means, const float *quats,
               const float *scales, const float *normals, const float *centroid,
               const float *colors_in, int64_t n, const dgsm_relight_params *params,
               float *colors_out, void *stream);

/* Pseudo-normals by local PCA (Sec. 4, lighting consistency: an alpha- and
 * distance-weighted PCA of the nearby Gaussian centres), for sh_relight's
 * `normals`.  For Gaussian i: the Gaussians j (i included) with
 * |x_j - x_i| <= radius, weighted w_j = opac_j (1 - |x_j - x_i|^2 / radius^2)^2;
 * the unit eigenvector of the smallest eigenvalue of their weighted
 * covariance; the smallest-scale axis of the Gaussian (first on ties) when
 * fewer than three neighbours carry weight or the covariance vanishes.  The
 * normal is flipped when n . (x_i - centroid) < 0.  means (n,3), opac (n),
 * quats (n,4; 16-byte aligned), scales (n,3), centroid (3), normals_out
 * (n,3): device.  0 <= n < 2^31, radius > 0 and finite.  Neighbours are found
 * through a spatial hash of cells of edge `radius` (workspace: about
 * 32 n + 16 max(2n, 1024) bytes).  Asynchronous. */
int dgsm_pca_normals(dgsm_ctx *ctx, const float *means, const float *opac, const float *quats,
                     const float *scales, int64_t n, float radius, const float *centroid,
                     float *normals_out, void *stream);

/* Storage order of a scene (a layout choice, not a step of Secs. 3.2-3.5:
 * every per-Gaussian result is independent of a Gaussian's place in the
 * arrays, and only the order of floating-point sums into an atlas voxel
 * changes).  perm_out (n int32, device) receives the permutation that sorts
 * the means (n,3; device) by their Z-order code on a 1024^3 grid over their
 * bounding box: cell q_a = floor((x_a - lo_a) * (1024 / (hi_a - lo_a)))
 * clamped to [0, 1023], each operation rounded once to float; code bit
 * 3b + a = bit b of q_a.  Equal codes keep their index order (stable).  A
 * flat axis, or a non-finite coordinate, gives cell 0 on that axis.  Stored
 * in this order, consecutive Gaussians are neighbours in space and in
 * direction from any light, so the atlas taps of a warp of receivers
 * (Sec. 3.3) share sectors.  0 <= n < 2^31; workspace about 16 n bytes.
 * Asynchronous. */
int dgsm_spatial_order(dgsm_ctx *ctx, const float *means, int64_t n, int32_t *perm_out, void *stream);

/* dst row i = src row perm[i] for i < n (rows of row_bytes bytes, a positive
 * multiple of 4; src holds n_src rows; src and dst device, 4-byte aligned,
 * distinct).  Applies a dgsm_spatial_order permutation to each attribute of
 * a scene.  A perm entry outside [0, n_src) leaves its row zero and records
 * DGSM_ERR_INVALID_ARG in the context's status word (dgsm_sync_status).
 * Asynchronous. */
int dgsm_gather_rows(dgsm_ctx *ctx, const void *src, int64_t n_src, int64_t row_bytes, const int32_t *perm,
                     int64_t n, void *dst, void *stream);

/* sh_relight for a Gaussian array made of n_obj contiguous objects (for
 * instance avatars): object o holds Gaussians [seg[o], seg[o+1]) and its
 * normals are turned away from centroids[o] (device, n_obj x 3 floats; see
 * dgsm_segment_centroids).  seg: HOST array of n_obj + 1 offsets with
 * seg[0] = 0, nondecreasing, seg[n_obj] = n; 1 <= n_obj <= 64 (read at the
 * call, so a captured graph keeps them). */
int sh_relight_objects(dgsm_ctx *ctx, const float *sh, const float *means, const float *quats,
                       const float *scales, const float *centroids, const int64_t *seg,
                       int32_t n_obj, const float *colors_in, int64_t n,
                       const dgsm_relight_params *params, float *colors_out, void *stream);

/* Alpha-weighted centroid of each object (the reference point of the relight
 * normals' orientation, Sec. 3.5): out[o] = sum_g w_g mean_g / sum_g w_g over
 * the object's Gaussians, summed in FP64 (0 for an empty or weightless
 * object).  means (n,3), weights (n) or NULL (weight 1): device; seg: host,
 * as for sh_relight_objects; out: device, n_obj x 3 floats. */
int dgsm_segment_centroids(dgsm_ctx *ctx, const float *means, const float *weights, int64_t n,
                           const int64_t *seg, int32_t n_obj, float *out, void *stream);

/* Rigid motion of whole objects: object o (Gaussians [seg[o], seg[o+1]))
 * moves by pose o = (qw, qx, qy, qz, tx, ty, tz, unused), the rotation
 * quaternion normalised here:  means_out = R(q_o) means + t,
 * quats_out = q_o * quats (Hamilton product, so R(quats_out) =
 * R(q_o) R(quats)); scales and opacities are unchanged.  means/quats (n,3)
 * and (n,4) device (quats 16-byte aligned); outputs may alias the inputs.
 * seg: host, as for sh_relight_objects.  poses: n_obj x 8 floats in device
 * memory or host memory (pinned when the call is captured in a graph); it
 * is copied on `stream`, so a replayed graph reads the poses present at
 * replay time. */
int dgsm_rigid_transform(dgsm_ctx *ctx, const float *means, const float *quats, int64_t n,
                         const int64_t *seg, int32_t n_obj, const float *poses, float *means_out,
                         float *quats_out, void *stream);

/* The moving-avatar frame (static scene + rigidly moving avatars, Secs.
 * 3.2-3.5) as ONE persistent cooperative kernel: every block stays resident
 * and the frame's steps are separated by grid-wide barriers instead of
 * kernel boundaries.  In order:
 *   1. rigid motion of the avatars to `poses` (as dgsm_rigid_transform);
 *   2. the avatars' dynamic atlases for all lights (as dgsm_build with
 *      tile 8 and params->max_pairs > 0: prep, the two binning levels, work
 *      items and the closed-form accumulation, Eqs. 3-4);
 *   3. every Gaussian, static then avatar, attenuated by
 *      T_static,l x T_dyn,l with light weights 1/L (as dgsm_attenuate_dyn);
 *   4. per-avatar alpha-weighted centroids (as dgsm_segment_centroids, the
 *      same FP64 sums in the same order) and the SH relight of the avatars
 *      (Eqs. 8-10, as sh_relight_objects).
 * Results equal those of the separate calls up to the order of floating-
 * point atomic sums in the atlas.  The launch (a memset of its barrier state
 * and one cooperative kernel) may be captured in a CUDA graph.
 *
 * Every barrier wait is bounded: a block that waits longer than about two
 * seconds (clock64 cycles at the SM clock) records DGSM_ERR_TIMEOUT in the
 * context's status word and returns, and so does every other block at its
 * next barrier; the context stays usable and the next call starts afresh.
 * timeout_barrier in 1..7 makes that barrier give up at once (a test of the
 * failure path); -1 (or any other value) for none.  The outputs of a frame
 * that timed out are incomplete.
 *
 * Arguments (all device pointers unless stated; float32):
 *   q_means (n_static + n_avatar, 3): the receivers; rows n_static.. are
 *     overwritten with the moved avatar means;
 *   colors_in, colors_out (n_static + n_avatar, 3);
 *   static_atlas [L][K][H][W] float32 with its radii (K floats);
 *   rest_means (n_avatar, 3), rest_quats (n_avatar, 4; 16-byte aligned),
 *     scales (n_avatar, 3), opac (n_avatar): the avatars at rest;
 *   quats_out (n_avatar, 4; 16-byte aligned): the moved rotations;
 *   seg: HOST array of n_obj + 1 offsets (as for sh_relight_objects);
 *   poses: n_obj x 8 floats, device or host (pinned when captured), copied
 *     on `stream` when the frame runs;
 *   dyn_atlas [L][K_dyn][H_dyn][W_dyn] float32 (written) with radii_dyn;
 *   lights (L, 3), 1 <= L <= 64; sh: 3 x 9 probe coefficients;
 *   centroids_out (n_obj, 3) (written); direct_frac as for dgsm_attenuate.
 * params: tile 8, atlas_dtype DGSM_F32, the octahedral map, max_pairs > 0
 * (capacity of both binning levels; a frame over it records
 * DGSM_ERR_WORKSPACE and leaves T_dyn = 1); L x super-tiles of the dynamic
 * atlas <= 4096 and L x tiles <= 65536.  Asynchronous; returns DGSM_OK,
 * DGSM_ERR_INVALID_ARG, DGSM_ERR_WORKSPACE (workspace would grow during a
 * capture) or DGSM_ERR_CUDA (the message names the call). */
typedef struct dgsm_crowd_frame_args {
    const float *q_means;
    const float *colors_in;
    float *colors_out;
    int64_t n_static;
    const float *static_atlas;
    int32_t H, W, K;
    const float *radii;
    const float *rest_means, *rest_quats, *scales, *opac;
    float *quats_out;
    int64_t n_avatar;
    const int64_t *seg;
    int32_t n_obj;
    const float *poses;
    float *dyn_atlas;
    int32_t H_dyn, W_dyn, K_dyn;
    const float *radii_dyn;
    const float *lights;
    int32_t L;
    const float *sh;
    float *centroids_out;
    float direct_frac;
} dgsm_crowd_frame_args;

int dgsm_crowd_frame(dgsm_ctx *ctx, const dgsm_crowd_frame_args *args, const dgsm_params *params,
                     const dgsm_relight_params *rparams, int32_t timeout_barrier, void *stream);

/* Phase times of the last dgsm_crowd_frame run while profiling was enabled
 * (dgsm_set_profiling): ms_out[0..7] (host) = the eight steps between the
 * kernel's start, its seven grid barriers and the last block's end, read from
 * the GPU's global timer.  Blocks.  Returns DGSM_ERR_INVALID_ARG when no
 * profiled frame ran. */
int dgsm_crowd_frame_phases(dgsm_ctx *ctx, double *ms_out);

/* CUDA-graph capture of library calls on `stream` (a created stream, not
 * the legacy default stream).  Between dgsm_graph_begin and dgsm_graph_end
 * only asynchronous calls may be made: dgsm_build with params->max_pairs > 0,
 * dgsm_attenuate, dgsm_rigid_transform, dgsm_segment_centroids, dgsm_crowd_frame,
 * sh_relight(_objects), sh_fit, dgsm_weighted_centroid, nf_attenuate.  The
 * context's workspace must already be large enough: make the same calls once
 * before capturing (a call that would grow it fails with
 * DGSM_ERR_WORKSPACE).  The graph keeps every pointer and size given at
 * capture: replay after changing buffer CONTENTS (and pinned host poses),
 * never the buffers themselves.  From dgsm_graph_begin until the graph is
 * destroyed the context's workspace does not grow; destroy the graph
 * before the context.  After a failed call inside the capture, still call
 * dgsm_graph_end (it then fails and returns no graph). */
int dgsm_graph_begin(dgsm_ctx *ctx, void *stream);
int dgsm_graph_end(dgsm_ctx *ctx, void *stream, dgsm_graph **out);
/* Replays the captured calls on `stream`; device-side errors land in the
 * context's status word (dgsm_sync_status). */
int dgsm_graph_launch(dgsm_graph *g, void *stream);
int dgsm_graph_node_count(dgsm_graph *g, int64_t *n_out);
void dgsm_graph_destroy(dgsm_graph *g);

/* Measured choice of the build's tile and chunk: runs dgsm_build once per
 * candidate (tiles[a], chunks[b]) to warm up, then `reps` timed runs (CUDA
 * events on `stream`); writes the median milliseconds to ms_out[a*n_chunks
 * + b] (host, may be NULL; -1 for a candidate the build rejects) and the
 * fastest parameters (base with that tile and chunk) to *best_out.  Writes
 * `atlas` as dgsm_build does.  Blocks. */
int dgsm_autotune_build(dgsm_ctx *ctx, const float *means, const float *scales,
                        const float *quats, const float *opac, int64_t n, const float *lights,
                        int32_t n_lights, int32_t H, int32_t W, const float *radii, int32_t K,
                        const dgsm_params *base, const int32_t *tiles, int32_t n_tiles,
                        const int32_t *chunks, int32_t n_chunks, int32_t reps, void *atlas,
                        dgsm_params *best_out, float *ms_out, void *stream);

/* Alpha-weighted centroid sum_i w_i mu_i / sum_i w_i of n Gaussians (the
 * receiver centroid the relight normals are turned away from, Sec. 3.2's
 * alpha-weighted avatar centroid), accumulated in FP64.  weights may be
 * NULL (plain mean); out: device pointer to 3 floats ((0,0,0) if the
 * weights sum to 0). */
int dgsm_weighted_centroid(dgsm_ctx *ctx, const float *means, const float *weights, int64_t n,
                           float *out, void *stream);

/* One frame from HOST memory: copy in, build the atlas from all n Gaussians
 * (dgsm_build), attenuate all n (dgsm_attenuate with one weight 1/L per light,
 * direct_frac 1), fit the probe (sh_fit), relight Gaussians
 * [relight_begin, relight_end) in place on their attenuated colours
 * (sh_relight, centroid = their alpha-weighted centroid), copy out.
 * All array fields of `in` are host pointers (pinned memory makes the copies
 * asynchronous); colors_out: host (n,3); sh_out: host (3,9) or NULL.
 * Device buffers come from the context's workspace.  The colours and the
 * cubemap are copied, and the probe is fitted, on a side stream of the
 * context while the build runs on `stream`; the colours outside the relit
 * range are copied back on it while the range is relit.  Blocks until the
 * results are in host memory. */
typedef struct {
    const float *means, *scales, *quats, *opac, *colors; /* (n,3) (n,3) (n,4) (n) (n,3) */
    int64_t n;
    int64_t relight_begin, relight_end;
    const float *lights;                                  /* (n_lights,3) */
    int32_t n_lights, H, W, K;
    const float *radii;                                   /* (K) */
    const float *cube_dirs, *cube_rgb, *cube_w;           /* (n_cube,3) (n_cube,3) (n_cube) */
    int64_t n_cube;
    double lambda;
} dgsm_frame_host_in;

int dgsm_frame_host(dgsm_ctx *ctx, const dgsm_frame_host_in *in, const dgsm_params *params,
                    const dgsm_relight_params *rparams, float *colors_out, float *sh_out,
                    void *stream);

/* dgsm_frame_host's frame, pipelined: submit returns once the frame is
 * enqueued (the build may block the host briefly to read its pair counts
 * when params->max_pairs is 0), so that a caller submitting frames to the two
 * slots in turn overlaps frame f's compute with the copy-in of frame f + 1
 * and the copy-out of frame f - 1.  The inputs go up on two copy streams of
 * the context at once; the compute runs on `stream` after everything
 * submitted there before (frames compute in submission order); the colours
 * come back on a copy-out stream.  Each slot (0 or 1) holds its own device
 * copies of the inputs, the atlas and the colours (context workspace); the
 * host arrays of `in`, colors_out and sh_out (pinned memory makes the copies
 * asynchronous) must stay valid and unchanged until dgsm_frame_host_wait on
 * the slot returns.  Submitting to a slot whose frame is in flight waits for
 * it first.  Returns DGSM_OK, DGSM_ERR_INVALID_ARG, DGSM_ERR_WORKSPACE or
 * DGSM_ERR_CUDA (enqueue errors); kernel errors of the frame come from the
 * wait. */
int dgsm_frame_host_submit(dgsm_ctx *ctx, int slot, const dgsm_frame_host_in *in, const dgsm_params *params,
                           const dgsm_relight_params *rparams, float *colors_out, float *sh_out,
                           void *stream);

/* Blocks until the slot's frame is complete (its colours and SH in host
 * memory) and returns the status its kernels recorded (DGSM_OK, or the
 * first error code); DGSM_OK at once for a slot with no frame in flight. */
int dgsm_frame_host_wait(dgsm_ctx *ctx, int slot);

/* Phase timing of dgsm_build.  While enabled, each dgsm_build records three
 * CUDA events on its stream (start; before the tile kernel; after it) for
 * up to 256 builds.  dgsm_profile_collect blocks until they complete and
 * writes, per build, ms_out[2b] = prep + binning + sort time and
 * ms_out[2b+1] = tile-kernel time (n_out builds), then forgets them. */
int dgsm_set_profiling(dgsm_ctx *ctx, int enable);
int dgsm_profile_collect(dgsm_ctx *ctx, double *ms_out, int max_builds, int *n_out);

/* ---- Learned transmittance surrogate (per-light neural field) ----------
 * A small network stands in for one light's atlas lookup: T_hat(u, v, rho) =
 * sigmoid(w5 . h4 + b5), h_l = ReLU(W_l h_{l-1} + b_l), four hidden layers of
 * width 64, h_0 = 96 Fourier features sin/cos(pi f_m x), f_m = 2^(8m/15),
 * m = 0..15, of x in {u, v, rho}: u, v the octahedral coordinates of the
 * direction (Eq. 6), rho = (k + w)/(K-1) the fractional shell coordinate of
 * the distance (as the trilinear lookup of Sec. 3.3 brackets it).  Features,
 * weights and hidden activations are bfloat16, sums float32 (tensor cores
 * for inference).  Parameters: one float32 vector of nf_param_count() values
 * per light: W1 [64][96], b1, W2 [64][64], b2, W3, b3, W4, b4, w5 [64], b5. */
int64_t nf_param_count(void);

/* Initial parameters: He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in))
 * drawn with SplitMix64 from (seed, index), zero biases. */
int nf_init(dgsm_ctx *ctx, uint64_t seed, float *params, void *stream);

/* Mean squared error of the field against `target` at the n inputs `uvr`
 * (n,3) and its gradient with respect to every parameter (float32,
 * nf_param_count() values); loss_out: device float or NULL.  n <= 2^24. */
int nf_loss_grad(dgsm_ctx *ctx, const float *params, const float *uvr, const float *target,
                 int64_t n, float *loss_out, float *grad_out, void *stream);

/* Adam training of one light's field on its exact atlas [K][H][W] (float32,
 * as dgsm_build writes it): every step draws `batch` voxels at random
 * (counter-based, from seed and the step number), fits T at the voxel
 * centres (u_j, v_i, k/(K-1)) by mean squared error, and updates params in
 * place (adam_m, adam_v: state of the same length, zero before the first
 * step).  step0: steps already taken (for bias correction when training is
 * resumed).  loss_out: `steps` floats (device) or NULL. */
int nf_train(dgsm_ctx *ctx, const float *atlas, int32_t H, int32_t W, int32_t K, float *params,
             float *adam_m, float *adam_v, int32_t steps, int32_t batch, float lr, uint64_t seed,
             int32_t step0, float *loss_out, void *stream);

/* Field values T_hat at n inputs (u, v, rho) (n,3) -> T_out (n). */
int nf_forward(dgsm_ctx *ctx, const float *params, const float *uvr, int64_t n, float *T_out,
               void *stream);

/* Largest |T_hat - T| over all voxels of each tile (tile x tile texels x K
 * shells) of one light's atlas [K][H][W]: tile_err (ceil(H/tile) *
 * ceil(W/tile) floats, row-major tiles).  Marks where the exact atlas must
 * stay as the fallback. */
int nf_tile_error(dgsm_ctx *ctx, const float *params, const float *atlas, int32_t H, int32_t W,
                  int32_t K, int32_t tile, float *tile_err, void *stream);

/* dgsm_attenuate with the field in place of the atlas lookup: params holds
 * n_lights parameter vectors back to back.  Where mask (n_lights x tiles,
 * uint8, nonzero = fall back) marks the tile of a query's texel cell, the
 * exact trilinear lookup in `atlas` ([n_lights][K][H][W] float32) is used
 * instead; mask and atlas may be NULL (field everywhere).  Other arguments
 * as for dgsm_attenuate.  The field runs on the tensor cores (tcgen05), one
 * light per CTA with its weights staged on chip; T of every (query, light)
 * goes through a context workspace of n_lights x n_q floats before the
 * colours are formed, so calls that share a context must share a stream. */
int nf_attenuate(dgsm_ctx *ctx, const float *params, const uint8_t *mask, const float *atlas,
                 int32_t n_lights, int32_t H, int32_t W, const float *radii, int32_t K,
                 int32_t tile, const float *lights, const float *q_means, const float *colors_in,
                 int64_t n_q, const float *light_w, float direct_frac, float *colors_out,
                 float *T_out, void *stream);

/* Measured single-precision ALU peaks of the context's GPU, the roofline
 * denominators of the build's tile kernel (its closed form of Eq. 3 is bound
 * by FP32 and special-function issue, not by memory).  out (host, 4
 * doubles): [0] FP32 fused multiply-add lane operations per second, [1]
 * ex2.approx, [2] rcp.approx, [3] rsqrt.approx lane operations per second.
 * Each comes from a kernel that fills every SM with independent dependency
 * chains of that one instruction, timed with CUDA events on `stream` (best
 * of three after one warm-up launch, about 0.5 s in all) at whatever SM
 * clock the GPU runs; nothing is changed on the GPU.  Blocks until done. */
int dgsm_measure_alu_peaks(dgsm_ctx *ctx, double *out, void *stream);

/* Reads and clears the context's device status word (blocks on `stream`):
 * returns DGSM_OK or the first error a kernel recorded since the last call. */
int dgsm_sync_status(dgsm_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DGSM_H */
