/*
 * dgsm_oracle.c -- plain, slow, FP64 CPU oracle for the Deep Gaussian Shadow
 * Map hot path (Sec. 3.2-3.5 of "Animated 3DGS Avatars in Diverse Scenes with
 * Consistent Lighting and Shadows").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; both sides only
 * take the same seeded inputs.
 *
 * Every floating-point quantity below is FP64 unless the function name says
 * f32: those few functions write out, in single precision with IEEE-rounded
 * operations in a fixed order, the integer decisions (texel, shell and tile
 * indices) that must come out bit-identical on the GPU.  This file must be
 * compiled without FMA contraction (-ffp-contract=off) and without
 * -ffast-math.
 *
 * Conventions (the paper leaves them open; the readings are ours):
 *   quaternion q = (w,x,y,z), normalised; R(q) the usual rotation matrix;
 *   Sigma = R diag(s^2) R^T with linear scales s; A = Sigma^-1.
 *   Atlas layout [L][K][H][W]; row i <-> v, column j <-> u; texel centres
 *   u_j = (2j+1)/W - 1, v_i = (2i+1)/H - 1; shell k holds T at t = r_k.
 *   sgn(0) = +1 in the octahedral fold.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ALPHA_MAX 0.999999  /* opacity clamp before tau* = -ln(1-alpha) */

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gaussian parameters (Sec. 3.2, problem statement and Eq. 5)               */
/* ------------------------------------------------------------------------ */

/* R(q) for q = (w,x,y,z); the quaternion is normalised first. */
void orc_quat_to_rot(const float *qf, double R[9]) {
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Precision A = Sigma^{-1} = R diag(1/s^2) R^T (Sec. 3.2). */
void orc_precision(const float *s, const float *q, double A[9]) {
    double R[9];
    orc_quat_to_rot(q, R);
    double inv[3] = {1.0 / ((double)s[0] * s[0]), 1.0 / ((double)s[1] * s[1]),
                     1.0 / ((double)s[2] * s[2])};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * inv[k] * R[3 * c + k];
            A[3 * r + c] = acc;
        }
}

/* Opacity-to-absorption mapping in use (ablation (B) of Sec. 4): 2 is Eq. 5.
 * Set for the whole library by orc_set_beta_mode (test infrastructure: one
 * mapping at a time). */
static int g_beta_mode = 2;
void orc_set_beta_mode(int mode) { g_beta_mode = mode; }
int orc_get_beta_mode(void) { return g_beta_mode; }

/* tau* = -ln(1-alpha) and
 *   mapping 1: beta = kappa tau*;
 *   mapping 2 (Eq. 5): beta = kappa tau* sqrt(tr(A)/3) / sqrt(2 pi), A the precision;
 *   mapping 3: beta = kappa tau* / ((2 pi)^(3/2) sqrt(det Sigma)), Sigma the covariance;
 *   mapping 4: beta = kappa tau* / ((2 pi)^(3/2) s_x s_y s_z).
 * det Sigma is taken from the covariance matrix itself (mapping 3) and from the
 * scales (mapping 4), so the two agree only up to rounding. */
double orc_beta(const float *s, float alpha, double kappa) {
    double a = alpha;
    if (!(a > 0)) return 0.0;
    if (a > ALPHA_MAX) a = ALPHA_MAX;
    double tau_star = -log1p(-a);
    double c = pow(2.0 * ORC_PI, 1.5);
    if (g_beta_mode == 1) return kappa * tau_star;
    if (g_beta_mode == 4) return kappa * tau_star / (c * (double)s[0] * s[1] * s[2]);
    double trA = 1.0 / ((double)s[0] * s[0]) + 1.0 / ((double)s[1] * s[1]) +
                 1.0 / ((double)s[2] * s[2]);
    return kappa * tau_star * sqrt(trA / 3.0) / sqrt(2.0 * ORC_PI);
}

/* Mapping 3 needs the rotation: sqrt(det Sigma) of Sigma = R diag(s^2) R^T
 * formed as a matrix and its determinant expanded by cofactors. */
static double beta_of(const float *s, const float *q, float alpha, double kappa) {
    if (g_beta_mode != 3) return orc_beta(s, alpha, kappa);
    double a = alpha;
    if (!(a > 0)) return 0.0;
    if (a > ALPHA_MAX) a = ALPHA_MAX;
    double tau_star = -log1p(-a);
    double R[9], S[9];
    orc_quat_to_rot(q, R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * ((double)s[k] * s[k]) * R[3 * c + k];
            S[3 * r + c] = acc;
        }
    double det = S[0] * (S[4] * S[8] - S[5] * S[7]) - S[1] * (S[3] * S[8] - S[5] * S[6]) +
                 S[2] * (S[3] * S[7] - S[4] * S[6]);
    return kappa * tau_star / (pow(2.0 * ORC_PI, 1.5) * sqrt(det));
}

/* Eq. 2 coefficients for the ray o + s d: a = d^T A d, b = d^T A (o-mu),
 * c = (o-mu)^T A (o-mu). */
void orc_ray_coeffs(const double A[9], const double *d, const double *o_minus_mu,
                    double *a, double *b, double *c) {
    double Ad[3], Aw[3];
    for (int r = 0; r < 3; ++r) {
        Ad[r] = A[3 * r] * d[0] + A[3 * r + 1] * d[1] + A[3 * r + 2] * d[2];
        Aw[r] = A[3 * r] * o_minus_mu[0] + A[3 * r + 1] * o_minus_mu[1] + A[3 * r + 2] * o_minus_mu[2];
    }
    *a = d[0] * Ad[0] + d[1] * Ad[1] + d[2] * Ad[2];
    *b = d[0] * Aw[0] + d[1] * Aw[1] + d[2] * Aw[2];
    *c = o_minus_mu[0] * Aw[0] + o_minus_mu[1] * Aw[1] + o_minus_mu[2] * Aw[2];
}

/* Eq. 3: int_0^t exp(-1/2 (a s^2 + 2 b s + c)) ds
 *   = sqrt(pi/(2a)) exp(-1/2 (c - b^2/a)) [erf(sqrt(a/2)(t + b/a)) - erf(sqrt(a/2) b/a)].
 * The erf difference is written with erfc so that it does not cancel when
 * both arguments lie far out on the same side. */
double orc_line_integral(double a, double b, double c, double t) {
    double m2 = c - b * b / a;
    if (m2 < 0) m2 = 0;  /* c - b^2/a >= 0 for positive definite A; rounding only */
    double pref = sqrt(ORC_PI / (2.0 * a)) * exp(-0.5 * m2);
    double h = sqrt(a / 2.0);
    double x0 = h * (b / a);
    double xt = h * (t + b / a);
    double diff;
    if (x0 >= 0)
        diff = erfc(x0) - erfc(xt);
    else if (xt <= 0)
        diff = erfc(-xt) - erfc(-x0);
    else
        diff = 2.0 - erfc(xt) - erfc(-x0);
    return pref * diff;
}

/* ------------------------------------------------------------------------ */
/* Octahedral map (Eq. 6 and its inverse, Sec. 3.2)                          */
/* ------------------------------------------------------------------------ */

static double sgn_pos(double x) { return x >= 0 ? 1.0 : -1.0; }

/* Eq. 6: q = d / (|x|+|y|+|z|); (u,v) = (qx,qy) if qz >= 0, else the fold. */
void orc_octa_encode(const double *d, double *u, double *v) {
    double l1 = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
    double qx = d[0] / l1, qy = d[1] / l1, qz = d[2] / l1;
    if (qz >= 0) {
        *u = qx; *v = qy;
    } else {
        *u = sgn_pos(qx) * (1.0 - fabs(qy));
        *v = sgn_pos(qy) * (1.0 - fabs(qx));
    }
}

/* Inverse: undo the fold, z = 1 - |u| - |v|, normalise. */
void orc_octa_decode(double u, double v, double *d) {
    double z = 1.0 - fabs(u) - fabs(v);
    double x = u, y = v;
    if (z < 0) {
        x = sgn_pos(u) * (1.0 - fabs(v));
        y = sgn_pos(v) * (1.0 - fabs(u));
    }
    double n = sqrt(x * x + y * y + z * z);
    d[0] = x / n; d[1] = y / n; d[2] = z / n;
}

/* Atlas parameterisation in use (ablation (C) of Sec. 4): 0 the octahedral
 * map, 1 a cube map of six F x F faces stacked in rows (H = 6F, W = F).  Set
 * for the whole library by orc_set_atlas_map (test infrastructure). */
static int g_atlas_map = 0;
void orc_set_atlas_map(int map) { g_atlas_map = map; }
int orc_get_atlas_map(void) { return g_atlas_map; }

/* Cube face f: forward axis, texel axes U (columns u) and V (rows v) as
 * (axis, sign): (+x, -z, -y), (-x, +z, -y), (+y, +x, +z), (-y, +x, -z),
 * (+z, +x, -y), (-z, -x, -y). */
static const int kCubeAxis[6][3] = {{0, 2, 1}, {0, 2, 1}, {1, 0, 2}, {1, 0, 2}, {2, 0, 1}, {2, 0, 1}};
static const int kCubeSign[6][3] = {{1, -1, -1}, {-1, 1, -1}, {1, 1, 1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, -1}};

/* Unit direction of the point (u, v) of cube face f. */
void orc_cube_decode(int f, double u, double v, double *d) {
    double c[3];
    c[kCubeAxis[f][0]] = kCubeSign[f][0];
    c[kCubeAxis[f][1]] = kCubeSign[f][1] * u;
    c[kCubeAxis[f][2]] = kCubeSign[f][2] * v;
    double n = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    d[0] = c[0] / n; d[1] = c[1] / n; d[2] = c[2] / n;
}

/* Face of the largest component (ties to x, then y; >= 0 the positive face)
 * and the face coordinates of d. */
int orc_cube_encode(const double *d, double *u, double *v) {
    double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
    int f = (ax >= ay && ax >= az) ? (d[0] >= 0 ? 0 : 1) : (ay >= az ? (d[1] >= 0 ? 2 : 3) : (d[2] >= 0 ? 4 : 5));
    double m = fabs(d[kCubeAxis[f][0]]);
    *u = kCubeSign[f][1] * d[kCubeAxis[f][1]] / m;
    *v = kCubeSign[f][2] * d[kCubeAxis[f][2]] / m;
    return f;
}

/* Direction of texel (i,j) of an H x W atlas: decode of its pixel centre
 * (octahedral, or face i / W of a cube map). */
void orc_texel_dir(int i, int j, int H, int W, double *d) {
    double u = (2.0 * j + 1.0) / W - 1.0;
    if (g_atlas_map == 1) {
        int f = i / W;
        double v = (2.0 * (i - f * W) + 1.0) / W - 1.0;
        orc_cube_decode(f, u, v, d);
        return;
    }
    double v = (2.0 * i + 1.0) / H - 1.0;
    orc_octa_decode(u, v, d);
}

/* ------------------------------------------------------------------------ */
/* DGSM build: brute force, every texel ray x every Gaussian x every shell   */
/* (Eqs. 1-5).  No culling, no window.                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    double A[9];
    double mu[3];
    double beta;
} orc_gauss;

static orc_gauss *prep_all(const float *means, const float *scales, const float *quats,
                           const float *opac, int64_t N, double kappa) {
    orc_gauss *g = (orc_gauss *)malloc(sizeof(orc_gauss) * (N > 0 ? N : 1));
    for (int64_t n = 0; n < N; ++n) {
        orc_precision(scales + 3 * n, quats + 4 * n, g[n].A);
        for (int c = 0; c < 3; ++c) g[n].mu[c] = means[3 * n + c];
        g[n].beta = beta_of(scales + 3 * n, quats + 4 * n, opac[n], kappa);
    }
    return g;
}

/* Optical depth tau(d, r_k) for one ray, all K shells (Eq. 2 summed with Eq. 3). */
static void ray_tau(const orc_gauss *g, int64_t N, const double *o, const double *d,
                    const float *radii, int K, double *tau) {
    for (int k = 0; k < K; ++k) tau[k] = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (g[n].beta == 0) continue;
        double om[3] = {o[0] - g[n].mu[0], o[1] - g[n].mu[1], o[2] - g[n].mu[2]};
        double a, b, c;
        orc_ray_coeffs(g[n].A, d, om, &a, &b, &c);
        for (int k = 0; k < K; ++k)
            tau[k] += g[n].beta * orc_line_integral(a, b, c, (double)radii[k]);
    }
}

/* Full atlas tau[l][k][i][j] (FP64).  Eq. 4 (T = exp(-tau)) is left to the
 * caller so that both tau and T are available. */
void orc_build_tau(const float *means, const float *scales, const float *quats,
                   const float *opac, int64_t N, const float *lights, int L, int H, int W,
                   const float *radii, int K, double kappa, double *tau_out) {
    orc_gauss *g = prep_all(means, scales, quats, opac, N, kappa);
    int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t idx = 0; idx < (int64_t)L * HW; ++idx) {
        int l = (int)(idx / HW);
        int i = (int)((idx % HW) / W), j = (int)(idx % W);
        double o[3] = {lights[3 * l], lights[3 * l + 1], lights[3 * l + 2]};
        double d[3], tau[512];
        orc_texel_dir(i, j, H, W, d);
        ray_tau(g, N, o, d, radii, K, tau);
        for (int k = 0; k < K; ++k) tau_out[((int64_t)l * K + k) * HW + (int64_t)i * W + j] = tau[k];
    }
    free(g);
}

/* tau for a list of texels (l,i,j), all K shells: tau_out[n][K]. */
void orc_build_tau_texels(const float *means, const float *scales, const float *quats,
                          const float *opac, int64_t N, const float *lights, int H, int W,
                          const float *radii, int K, double kappa, const int32_t *lij,
                          int64_t n_texels, double *tau_out) {
    orc_gauss *g = prep_all(means, scales, quats, opac, N, kappa);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < n_texels; ++t) {
        int l = lij[3 * t], i = lij[3 * t + 1], j = lij[3 * t + 2];
        double o[3] = {lights[3 * l], lights[3 * l + 1], lights[3 * l + 2]};
        double d[3];
        orc_texel_dir(i, j, H, W, d);
        ray_tau(g, N, o, d, radii, K, tau_out + t * K);
    }
    free(g);
}

/* tau along arbitrary rays (origin o_l of light l, unit direction d) at
 * arbitrary distances t: used by the quadrature pins. */
void orc_tau_rays(const float *means, const float *scales, const float *quats,
                  const float *opac, int64_t N, const double *origins, const double *dirs,
                  const double *t, int64_t n_rays, double kappa, double *tau_out) {
    orc_gauss *g = prep_all(means, scales, quats, opac, N, kappa);
    for (int64_t r = 0; r < n_rays; ++r) {
        double acc = 0;
        for (int64_t n = 0; n < N; ++n) {
            if (g[n].beta == 0) continue;
            double om[3] = {origins[3 * r] - g[n].mu[0], origins[3 * r + 1] - g[n].mu[1],
                            origins[3 * r + 2] - g[n].mu[2]};
            double a, b, c;
            orc_ray_coeffs(g[n].A, dirs + 3 * r, om, &a, &b, &c);
            acc += g[n].beta * orc_line_integral(a, b, c, t[r]);
        }
        tau_out[r] = acc;
    }
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Sampling (Sec. 3.3): centre lookup with trilinear interpolation           */
/* ------------------------------------------------------------------------ */

/* Continuous lookup of one light's atlas T[K][H][W] (FP64) at world point x:
 * bilinear between texel centres with clamp-to-edge, linear between the two
 * shells bracketing t (k = #{r_k <= t} - 1, clamped at both ends). */
double orc_sample_T(const double *atlas_l, int H, int W, const float *radii, int K,
                    const double *o, const double *x) {
    double vx = x[0] - o[0], vy = x[1] - o[1], vz = x[2] - o[2];
    double t = sqrt(vx * vx + vy * vy + vz * vz);
    if (t == 0) return 1.0;
    double d[3] = {vx / t, vy / t, vz / t}, u, v;
    int r0 = 0, hf = H;   /* rows of the point's face (all rows for the octahedral map) */
    if (g_atlas_map == 1) {
        int f = orc_cube_encode(d, &u, &v);
        r0 = f * W;
        hf = W;
    } else {
        orc_octa_encode(d, &u, &v);
    }
    double gx = (u + 1.0) * 0.5 * W - 0.5, gy = (v + 1.0) * 0.5 * hf - 0.5;
    double fj = floor(gx), fi = floor(gy);
    double ax = gx - fj, ay = gy - fi;
    int j0 = (int)fj, i0 = (int)fi, j1 = j0 + 1, i1 = i0 + 1;
    if (j0 < 0) j0 = 0; if (j0 > W - 1) j0 = W - 1;
    if (j1 < 0) j1 = 0; if (j1 > W - 1) j1 = W - 1;
    if (i0 < 0) i0 = 0; if (i0 > hf - 1) i0 = hf - 1;
    if (i1 < 0) i1 = 0; if (i1 > hf - 1) i1 = hf - 1;
    i0 += r0;
    i1 += r0;
    int k = -1;
    for (int q = 0; q < K; ++q)
        if ((double)radii[q] <= t) k = q;
    int k0, k1;
    double wt;
    if (k < 0) { k0 = k1 = 0; wt = 0; }
    else if (k >= K - 1) { k0 = k1 = K - 1; wt = 0; }
    else { k0 = k; k1 = k + 1; wt = (t - radii[k]) / ((double)radii[k + 1] - radii[k]); }
    int64_t HW = (int64_t)H * W;
    double res = 0;
    for (int s = 0; s < 2; ++s) {
        int kk = s ? k1 : k0;
        double ws = s ? wt : 1.0 - wt;
        const double *P = atlas_l + (int64_t)kk * HW;
        double b = (1 - ay) * ((1 - ax) * P[(int64_t)i0 * W + j0] + ax * P[(int64_t)i0 * W + j1]) +
                   ay * ((1 - ax) * P[(int64_t)i1 * W + j0] + ax * P[(int64_t)i1 * W + j1]);
        res += ws * b;
    }
    return res;
}

/* Attenuation of receivers (Sec. 3.3): the direct part of each colour is
 * scaled by the light-weighted transmittance,
 *   c' = c (1 - w_d + w_d sum_l omega_l T_l(x)),
 * with T_l = T_static,l * T_dynamic,l when a second atlas is given.
 * atlas: [L][K][H][W] FP64; atlas_dyn may be NULL; light_w may be NULL (1/L). */
void orc_attenuate(const double *atlas, const double *atlas_dyn, int L, int H, int W,
                   const float *radii, int K, const float *lights, const float *q_means,
                   const float *colors_in, int64_t Q, const float *light_w, double direct_frac,
                   double *colors_out, double *T_out) {
    int64_t LS = (int64_t)K * H * W;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < Q; ++q) {
        double x[3] = {q_means[3 * q], q_means[3 * q + 1], q_means[3 * q + 2]};
        double acc = 0;
        for (int l = 0; l < L; ++l) {
            double o[3] = {lights[3 * l], lights[3 * l + 1], lights[3 * l + 2]};
            double T = orc_sample_T(atlas + l * LS, H, W, radii, K, o, x);
            if (atlas_dyn) T *= orc_sample_T(atlas_dyn + l * LS, H, W, radii, K, o, x);
            if (T_out) T_out[q * L + l] = T;
            double wl = light_w ? (double)light_w[l] : 1.0 / L;
            acc += wl * T;
        }
        double f = 1.0 - direct_frac + direct_frac * acc;
        for (int c = 0; c < 3; ++c) colors_out[3 * q + c] = (double)colors_in[3 * q + c] * f;
    }
}

/* ------------------------------------------------------------------------ */
/* FP32 index specification (bit-exact decisions shared with the GPU)        */
/* ------------------------------------------------------------------------ */

static float sgnf_pos(float x) { return x >= 0.0f ? 1.0f : -1.0f; }

/* Texel cell, bilinear base tap and shell of the world point x seen from o.
 * out_i[0..4] = cell i, cell j, bilinear base i0, base j0, shell k (-1 below r_0);
 * out_f[0..2] = fy, fx (bilinear fractions), t (distance).  All single
 * precision, IEEE-rounded, no FMA. */
static void f32_sample_index_cube(const float *x, const float *o, int F, const float *radii, int K,
                                  int32_t *out_i, float *out_f);

void orc_f32_sample_index(const float *x, const float *o, int H, int W, const float *radii,
                          int K, int32_t *out_i, float *out_f) {
    if (g_atlas_map == 1) {
        f32_sample_index_cube(x, o, W, radii, K, out_i, out_f);
        return;
    }
    volatile float vx = x[0] - o[0], vy = x[1] - o[1], vz = x[2] - o[2];
    volatile float t2a = vx * vx, t2b = vy * vy, t2c = vz * vz;
    volatile float t2 = (t2a + t2b) + t2c;
    float t = sqrtf(t2);
    volatile float s = (fabsf(vx) + fabsf(vy)) + fabsf(vz);
    float u, v;
    if (s == 0.0f) { u = 0.0f; v = 0.0f; }
    else {
        volatile float qx = vx / s, qy = vy / s;
        if (vz >= 0.0f) { u = qx; v = qy; }
        else {
            volatile float a = 1.0f - fabsf(qy), b = 1.0f - fabsf(qx);
            u = sgnf_pos(qx) * a; v = sgnf_pos(qy) * b;
        }
    }
    volatile float fu = ((u + 1.0f) * 0.5f) * (float)W;
    volatile float fv = ((v + 1.0f) * 0.5f) * (float)H;
    volatile float gx = fu - 0.5f, gy = fv - 0.5f;
    float bj = floorf(gx), bi = floorf(gy);
    int cj = (int)floorf(fu), ci = (int)floorf(fv);
    if (cj < 0) cj = 0; if (cj > W - 1) cj = W - 1;
    if (ci < 0) ci = 0; if (ci > H - 1) ci = H - 1;
    int k = -1;
    for (int q = 0; q < K; ++q)
        if (radii[q] <= t) k = q;
    out_i[0] = ci; out_i[1] = cj; out_i[2] = (int32_t)bi; out_i[3] = (int32_t)bj; out_i[4] = k;
    volatile float fy = gy - bi, fx = gx - bj;
    out_f[0] = fy; out_f[1] = fx; out_f[2] = t;
}

/* The same decisions on a cube map of F x F faces (rows global, face f's
 * rows from f F): the face of the largest component of v = x - o (ties to x,
 * then y; a component >= 0 picks the positive face), u = U.v / m,
 * v = V.v / m with m that component's size, then as for the octahedral map
 * within the face. */
static void f32_sample_index_cube(const float *x, const float *o, int F, const float *radii, int K,
                                  int32_t *out_i, float *out_f) {
    volatile float vx = x[0] - o[0], vy = x[1] - o[1], vz = x[2] - o[2];
    volatile float t2a = vx * vx, t2b = vy * vy, t2c = vz * vz;
    volatile float t2 = (t2a + t2b) + t2c;
    float t = sqrtf(t2);
    float c[3] = {vx, vy, vz};
    float ax = fabsf(c[0]), ay = fabsf(c[1]), az = fabsf(c[2]);
    int f = (ax >= ay && ax >= az) ? (c[0] >= 0.0f ? 0 : 1) : (ay >= az ? (c[1] >= 0.0f ? 2 : 3) : (c[2] >= 0.0f ? 4 : 5));
    float m = fabsf(c[kCubeAxis[f][0]]);
    float u = 0.0f, v = 0.0f;
    if (m != 0.0f) {
        volatile float nu = (float)kCubeSign[f][1] * c[kCubeAxis[f][1]];
        volatile float nv = (float)kCubeSign[f][2] * c[kCubeAxis[f][2]];
        volatile float qu = nu / m, qv = nv / m;
        u = qu;
        v = qv;
    }
    volatile float fu = ((u + 1.0f) * 0.5f) * (float)F;
    volatile float fv = ((v + 1.0f) * 0.5f) * (float)F;
    volatile float gx = fu - 0.5f, gy = fv - 0.5f;
    float bj = floorf(gx), bi = floorf(gy);
    int cj = (int)floorf(fu), ci = (int)floorf(fv);
    if (cj < 0) cj = 0; if (cj > F - 1) cj = F - 1;
    if (ci < 0) ci = 0; if (ci > F - 1) ci = F - 1;
    int k = -1;
    for (int q = 0; q < K; ++q)
        if (radii[q] <= t) k = q;
    out_i[0] = f * F + ci; out_i[1] = cj; out_i[2] = f * F + (int32_t)bi; out_i[3] = (int32_t)bj; out_i[4] = k;
    volatile float fy = gy - bi, fx = gx - bj;
    out_f[0] = fy; out_f[1] = fx; out_f[2] = t;
}

void orc_f32_sample_index_batch(const float *x, int64_t n, const float *o, int H, int W,
                                const float *radii, int K, int32_t *out_i, float *out_f) {
    for (int64_t q = 0; q < n; ++q)
        orc_f32_sample_index(x + 3 * q, o, H, W, radii, K, out_i + 5 * q, out_f + 3 * q);
}

/* FP32 decode of an atlas point (u,v), normalised. */
static void f32_decode(float u, float v, float *d) {
    volatile float au = fabsf(u), av = fabsf(v);
    volatile float z = (1.0f - au) - av;
    volatile float x = u, y = v;
    if (z < 0.0f) {
        volatile float a = 1.0f - av, b = 1.0f - au;
        x = sgnf_pos(u) * a;
        y = sgnf_pos(v) * b;
    }
    volatile float xx = x * x, yy = y * y, zz = z * z;
    volatile float n2 = (xx + yy) + zz;
    float n = sqrtf(n2);
    volatile float dx = x / n, dy = y / n, dz = z / n;
    d[0] = dx; d[1] = dy; d[2] = dz;
}

static float f32_dot(const float *a, const float *b) {
    volatile float p0 = a[0] * b[0], p1 = a[1] * b[1], p2 = a[2] * b[2];
    volatile float s = p0 + p1;
    volatile float r = s + p2;
    return r;
}

/* Texel-centre coordinate of index j in an extent of W texels, FP32. */
static float f32_centre(int j, int W) {
    volatile float num = (float)(2 * j + 1);
    volatile float q = num / (float)W;
    volatile float r = q - 1.0f;
    return r;
}

/* FP32 decode of the point (u, v) of cube face f, normalised. */
static void f32_decode_cube(int f, float u, float v, float *d) {
    float c[3];
    c[kCubeAxis[f][0]] = (float)kCubeSign[f][0];
    c[kCubeAxis[f][1]] = (float)kCubeSign[f][1] * u;
    c[kCubeAxis[f][2]] = (float)kCubeSign[f][2] * v;
    volatile float xx = c[0] * c[0], yy = c[1] * c[1], zz = c[2] * c[2];
    volatile float n2 = (xx + yy) + zz;
    float n = sqrtf(n2);
    volatile float dx = c[0] / n, dy = c[1] / n, dz = c[2] / n;
    d[0] = dx; d[1] = dy; d[2] = dz;
}

/* Cone of a rectangle of a cube-map atlas (faces of F = W texels stacked in
 * rows).  Its part on one face is a convex spherical quadrilateral (the
 * decode is a central projection of the face plane), so a cap of half-angle
 * below 90 degrees holds the part iff it holds its four corners.  Axis: the
 * decoded centre of a rectangle on one face; the normalised sum of the
 * decoded centres of its parts for one across faces.  Half-angle: the
 * largest angle to a corner of any part. */
static void f32_rect_cone_cube(int i0, int i1, int j0, int j1, int F, float *cone) {
    int f0 = i0 / F, f1 = (i1 - 1) / F;
    float ua = f32_centre(j0, F), ub = f32_centre(j1 - 1, F);
    volatile float su = ua + ub;
    volatile float uc = su * 0.5f;
    float c[3];
    if (f0 == f1) {
        float va = f32_centre(i0 - f0 * F, F), vb = f32_centre(i1 - 1 - f0 * F, F);
        volatile float sv = va + vb;
        volatile float vc = sv * 0.5f;
        f32_decode_cube(f0, uc, vc, c);
    } else {
        volatile float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        for (int f = f0; f <= f1; ++f) {
            int r0 = (i0 > f * F ? i0 : f * F) - f * F;
            int r1 = (i1 < (f + 1) * F ? i1 : (f + 1) * F) - 1 - f * F;
            float va = f32_centre(r0, F), vb = f32_centre(r1, F);
            volatile float sv = va + vb;
            volatile float vc = sv * 0.5f;
            float d[3];
            f32_decode_cube(f, uc, vc, d);
            sx = sx + d[0];
            sy = sy + d[1];
            sz = sz + d[2];
        }
        volatile float xx = sx * sx, yy = sy * sy, zz = sz * sz;
        volatile float n2 = (xx + yy) + zz;
        float n = sqrtf(n2);
        if (!(n > 0.0f)) {
            cone[0] = 0.0f; cone[1] = 0.0f; cone[2] = 1.0f; cone[3] = -1.0f; cone[4] = 0.0f; cone[5] = 1.0f;
            return;
        }
        volatile float cx = sx / n, cy = sy / n, cz = sz / n;
        c[0] = cx; c[1] = cy; c[2] = cz;
    }
    float us[2] = {ua, ub}, cmin = 1.0f;
    for (int f = f0; f <= f1; ++f) {
        int r0 = (i0 > f * F ? i0 : f * F) - f * F;
        int r1 = (i1 < (f + 1) * F ? i1 : (f + 1) * F) - 1 - f * F;
        float vs[2] = {f32_centre(r0, F), f32_centre(r1, F)};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                float d[3];
                f32_decode_cube(f, us[b], vs[a], d);
                float cs = f32_dot(c, d);
                if (cs < cmin) cmin = cs;
            }
    }
    cone[0] = c[0]; cone[1] = c[1]; cone[2] = c[2];
    if (cmin <= 0.0f) {
        cone[3] = -1.0f; cone[4] = 0.0f; cone[5] = 1.0f;
    } else {
        volatile float cc = cmin * cmin;
        volatile float om = 1.0f - cc;
        cone[3] = cmin; cone[4] = sqrtf(om); cone[5] = 0.0f;
    }
}

/* Direction cone of the texel-centre rectangle [j0,j1) x [i0,i1):
 * cone[0..2] axis, cone[3] cos, cone[4] sin, cone[5] = 1 if it spans a
 * hemisphere or more (then every Gaussian overlaps it). */
void orc_f32_rect_cone(int i0, int i1, int j0, int j1, int H, int W, float *cone) {
    if (g_atlas_map == 1) {
        f32_rect_cone_cube(i0, i1, j0, j1, W, cone);
        return;
    }
    float ua = f32_centre(j0, W), ub = f32_centre(j1 - 1, W);
    float va = f32_centre(i0, H), vb = f32_centre(i1 - 1, H);
    volatile float su = ua + ub, sv = va + vb;
    volatile float uc = su * 0.5f, vc = sv * 0.5f;
    float c[3];
    f32_decode(uc, vc, c);
    float pts[64][2];
    int np = 0;
    pts[np][0] = ua; pts[np][1] = va; ++np;
    pts[np][0] = ub; pts[np][1] = va; ++np;
    pts[np][0] = ua; pts[np][1] = vb; ++np;
    pts[np][0] = ub; pts[np][1] = vb; ++np;
    float ve[2] = {va, vb}, ue[2] = {ua, ub};
    for (int e = 0; e < 2; ++e) {
        volatile float y = ve[e];
        volatile float cand[5];
        cand[0] = 0.0f; cand[1] = 1.0f - y; cand[2] = -1.0f - y; cand[3] = 1.0f + y; cand[4] = y - 1.0f;
        for (int m = 0; m < 5; ++m)
            if (ua <= cand[m] && cand[m] <= ub) { pts[np][0] = cand[m]; pts[np][1] = y; ++np; }
    }
    for (int e = 0; e < 2; ++e) {
        volatile float xx = ue[e];
        volatile float cand[5];
        cand[0] = 0.0f; cand[1] = 1.0f - xx; cand[2] = -1.0f - xx; cand[3] = 1.0f + xx; cand[4] = xx - 1.0f;
        for (int m = 0; m < 5; ++m)
            if (va <= cand[m] && cand[m] <= vb) { pts[np][0] = xx; pts[np][1] = cand[m]; ++np; }
    }
    if (ua <= 0.0f && 0.0f <= ub && va <= 0.0f && 0.0f <= vb) { pts[np][0] = 0.0f; pts[np][1] = 0.0f; ++np; }
    float cmin = 1.0f;
    for (int p = 0; p < np; ++p) {
        float d[3];
        f32_decode(pts[p][0], pts[p][1], d);
        float cs = f32_dot(c, d);
        if (cs < cmin) cmin = cs;
    }
    cone[0] = c[0]; cone[1] = c[1]; cone[2] = c[2];
    if (cmin <= 0.0f) {
        cone[3] = -1.0f; cone[4] = 0.0f; cone[5] = 1.0f;
    } else {
        volatile float cc = cmin * cmin;
        volatile float om = 1.0f - cc;
        cone[3] = cmin; cone[4] = sqrtf(om); cone[5] = 0.0f;
    }
}

/* Per-(light, Gaussian) bounding cone of the binning specification.
 * out[0..2] unit direction to the Gaussian, out[3] cos, out[4] sin,
 * out[5] = 1 if the light lies inside the bounding sphere (all tiles),
 * out[6] = k^2 (cull radius in Mahalanobis units), out[7] = sphere radius r,
 * out[8] = distance. Returns 0 if the Gaussian is binned nowhere (alpha <= 0,
 * or wholly beyond the last shell), 1 otherwise, -1 on invalid input. */
int orc_f32_gauss_cone(const float *mu, const float *s, float alpha, const float *o,
                       float kappa, float eps, float r_last, float *out) {
    for (int c = 0; c < 3; ++c)
        if (!isfinite(mu[c]) || !isfinite(s[c]) || !(s[c] > 0.0f)) return -1;
    if (!isfinite(alpha)) return -1;
    float a = alpha;
    if (!(a > 0.0f)) return 0;
    if (a > 0.999999f) a = 0.999999f;
    float smax = fmaxf(fmaxf(s[0], s[1]), s[2]);
    float smin = fminf(fminf(s[0], s[1]), s[2]);
    volatile float om = 1.0f - a;
    volatile float odds = a / om;
    volatile float t1 = kappa * odds;
    /* bound of beta sqrt(2 pi / a) / tau* along any ray, per mapping */
    volatile float ratio;
    if (g_beta_mode == 1) {
        ratio = 2.50662827f * smax;
    } else if (g_beta_mode == 3 || g_beta_mode == 4) {
        volatile float p01 = s[0] * s[1];
        volatile float p012 = p01 * s[2];
        volatile float den = 6.28318531f * p012;
        ratio = smax / den;
    } else {
        ratio = smax / smin;
    }
    volatile float t2 = t1 * ratio;
    volatile float Q = t2 / eps;
    int e = 0;
    frexpf(Q, &e);
    if (e < 1) e = 1;
    volatile float k2 = 1.38629436f * (float)e;
    volatile float k = sqrtf(k2);
    volatile float r = k * smax;
    volatile float vx = mu[0] - o[0], vy = mu[1] - o[1], vz = mu[2] - o[2];
    volatile float xx = vx * vx, yy = vy * vy, zz = vz * vz;
    volatile float d2 = (xx + yy) + zz;
    float dist = sqrtf(d2);
    volatile float lo = dist - r;
    out[6] = k2; out[7] = r; out[8] = dist;
    if (lo > r_last) return 0;
    if (r >= dist) {
        out[0] = 0; out[1] = 0; out[2] = 1; out[3] = -1.0f; out[4] = 0.0f; out[5] = 1.0f;
        return 1;
    }
    volatile float sn = r / dist;
    volatile float sn2 = sn * sn;
    volatile float c2 = 1.0f - sn2;
    out[0] = vx / dist; out[1] = vy / dist; out[2] = vz / dist;
    out[3] = sqrtf(c2); out[4] = sn; out[5] = 0.0f;
    return 1;
}

/* Cone-cone overlap: angle(dir, axis) <= theta_g + theta_T, evaluated as
 * dir . axis >= cos_g cos_T - sin_g sin_T. */
static int f32_overlap(const float *g, const float *cone) {
    if (g[5] != 0.0f || cone[5] != 0.0f) return 1;
    float dot = f32_dot(g, cone);
    volatile float p = g[3] * cone[3], q = g[4] * cone[4];
    volatile float rhs = p - q;
    return dot >= rhs;
}

static void f32_cross(const float *a, const float *b, float *c) {
    volatile float p0 = a[1] * b[2], q0 = a[2] * b[1];
    volatile float p1 = a[2] * b[0], q1 = a[0] * b[2];
    volatile float p2 = a[0] * b[1], q2 = a[1] * b[0];
    volatile float c0 = p0 - q0, c1 = p1 - q1, c2 = p2 - q2;
    c[0] = c0; c[1] = c1; c[2] = c2;
}

/* Octahedral face of an atlas point: bit 0 u >= 0, bit 1 v >= 0, bit 2 the
 * upper hemisphere ((1 - |u|) - |v| >= 0, as f32_decode decides it). */
static int f32_face(float u, float v) {
    volatile float au = fabsf(u), av = fabsf(v);
    volatile float z = (1.0f - au) - av;
    return (u >= 0.0f ? 1 : 0) | (v >= 0.0f ? 2 : 0) | (z >= 0.0f ? 4 : 0);
}

/* Plane through the light containing directions a and b, oriented so that
 * direction c lies on its non-negative side. */
static void f32_plane(const float *a, const float *b, const float *c, float *n) {
    f32_cross(a, b, n);
    if (f32_dot(n, c) < 0.0f) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
}

/* Separating planes of the texel-centre rectangle [j0,j1) x [i0,i1) for the
 * ellipsoid test of the binning specification.  Inside one octahedral face
 * the decode is affine in (u,v), so lines of the atlas are great circles and
 * the rays through the rectangle's texel centres lie in the polyhedral cone
 * of its four corner directions.  pl[0..2] top edge (row i0), [3..5] bottom
 * edge (row i1-1), [6..8] left (column j0), [9..11] right (column j1-1),
 * [12..14] the plane between the halves (rows [i0, i0+half) and
 * [i0+half, i1)), each oriented non-negative on the rectangle's side (the
 * mid plane: on the top half's side); pl[15] = 1 if the planes are valid
 * (the rectangle lies in one face and has at least 2 rows and 2 columns);
 * pl[16] = 1 if the bottom half is not empty. */
static void f32_rect_planes_cube(int i0, int i1, int j0, int j1, int half, int F, float *pl);

void orc_f32_rect_planes(int i0, int i1, int j0, int j1, int half, int H, int W, float *pl) {
    if (g_atlas_map == 1) {
        f32_rect_planes_cube(i0, i1, j0, j1, half, W, pl);
        return;
    }
    float ua = f32_centre(j0, W), ub = f32_centre(j1 - 1, W);
    float va = f32_centre(i0, H), vb = f32_centre(i1 - 1, H);
    for (int q = 0; q < 17; ++q) pl[q] = 0.0f;
    pl[16] = i1 - i0 > half ? 1.0f : 0.0f;
    int f = f32_face(ua, va);
    if (!(ua < ub && va < vb) || f32_face(ub, va) != f || f32_face(ua, vb) != f || f32_face(ub, vb) != f)
        return;
    volatile float su = ua + ub, sv = va + vb;
    volatile float uc = su * 0.5f, vc = sv * 0.5f;
    float c[3], d00[3], d01[3], d10[3], d11[3];
    f32_decode(uc, vc, c);
    f32_decode(ua, va, d00); f32_decode(ub, va, d01);
    f32_decode(ua, vb, d10); f32_decode(ub, vb, d11);
    f32_plane(d00, d01, c, pl);
    f32_plane(d10, d11, c, pl + 3);
    f32_plane(d00, d10, c, pl + 6);
    f32_plane(d01, d11, c, pl + 9);
    if (pl[16] != 0.0f) {
        volatile float num = (float)(2 * (i0 + half));
        volatile float q = num / (float)H;
        volatile float vm = q - 1.0f;
        float m0[3], m1[3], top[3];
        f32_decode(ua, vm, m0); f32_decode(ub, vm, m1);
        f32_decode(uc, va, top);
        f32_plane(m0, m1, top, pl + 12);
    }
    pl[15] = 1.0f;
}

/* Planes of a rectangle of a cube-map atlas: the edge planes through its
 * corner directions and the plane between its halves (atlas lines are great
 * circles within a face). */
static void f32_rect_planes_cube(int i0, int i1, int j0, int j1, int half, int F, float *pl) {
    int f = i0 / F;
    float ua = f32_centre(j0, F), ub = f32_centre(j1 - 1, F);
    float va = f32_centre(i0 - f * F, F), vb = f32_centre(i1 - 1 - f * F, F);
    for (int q = 0; q < 17; ++q) pl[q] = 0.0f;
    pl[16] = i1 - i0 > half ? 1.0f : 0.0f;
    if (!(ua < ub && va < vb) || (i1 - 1) / F != f) return;
    volatile float su = ua + ub, sv = va + vb;
    volatile float uc = su * 0.5f, vc = sv * 0.5f;
    float c[3], d00[3], d01[3], d10[3], d11[3];
    f32_decode_cube(f, uc, vc, c);
    f32_decode_cube(f, ua, va, d00); f32_decode_cube(f, ub, va, d01);
    f32_decode_cube(f, ua, vb, d10); f32_decode_cube(f, ub, vb, d11);
    f32_plane(d00, d01, c, pl);
    f32_plane(d10, d11, c, pl + 3);
    f32_plane(d00, d10, c, pl + 6);
    f32_plane(d01, d11, c, pl + 9);
    if (pl[16] != 0.0f) {
        volatile float num = (float)(2 * (i0 + half - f * F));
        volatile float q = num / (float)F;
        volatile float vm = q - 1.0f;
        float m0[3], m1[3], top[3];
        f32_decode_cube(f, ua, vm, m0); f32_decode_cube(f, ub, vm, m1);
        f32_decode_cube(f, uc, va, top);
        f32_plane(m0, m1, top, pl + 12);
    }
    pl[15] = 1.0f;
}

/* Axes of a Gaussian for the ellipsoid test: out[0..2] = v = mu - o and
 * out[3+3k .. 5+3k] = s_k times column k of R(q) (q normalised), so that
 * n^T Sigma n = sum_k ((s_k r_k) . n)^2 -- a sum of squares, exact in sign
 * for flat Gaussians. */
void orc_f32_gauss_axes(const float *mu, const float *s, const float *q, const float *o, float *out) {
    volatile float vx = mu[0] - o[0], vy = mu[1] - o[1], vz = mu[2] - o[2];
    volatile float ww = q[0] * q[0], xx = q[1] * q[1], yy = q[2] * q[2], zz = q[3] * q[3];
    volatile float n2a = ww + xx;
    volatile float n2b = n2a + yy;
    volatile float n2 = n2b + zz;
    float n = sqrtf(n2);
    volatile float w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    volatile float pxx = x * x, pyy = y * y, pzz = z * z;
    volatile float pxy = x * y, pxz = x * z, pyz = y * z;
    volatile float pwx = w * x, pwy = w * y, pwz = w * z;
    volatile float t00 = pyy + pzz, t11 = pxx + pzz, t22 = pxx + pyy;
    volatile float t01 = pxy - pwz, t10 = pxy + pwz, t02 = pxz + pwy;
    volatile float t20 = pxz - pwy, t12 = pyz - pwx, t21 = pyz + pwx;
    volatile float u00 = 2.0f * t00, u11 = 2.0f * t11, u22 = 2.0f * t22;
    float R[9];
    volatile float r00 = 1.0f - u00, r11 = 1.0f - u11, r22 = 1.0f - u22;
    volatile float r01 = 2.0f * t01, r10 = 2.0f * t10, r02 = 2.0f * t02;
    volatile float r20 = 2.0f * t20, r12 = 2.0f * t12, r21 = 2.0f * t21;
    R[0] = r00; R[1] = r01; R[2] = r02; R[3] = r10; R[4] = r11; R[5] = r12; R[6] = r20; R[7] = r21; R[8] = r22;
    out[0] = vx; out[1] = vy; out[2] = vz;
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) {
            volatile float e = R[3 * r + k] * s[k];
            out[3 + 3 * k + r] = e;
        }
}

/* Does the Gaussian's culling ellipsoid {x : (x-mu)^T A (x-mu) <= k^2}
 * reach the non-negative side of plane n?  Its support there is
 * n.v + k sqrt(n^T Sigma n); the test compares squares (with k^2 widened by
 * 2^-10 against rounding) when n.v < 0. */
/* Dot product of the plane tests: a0 b0, then fused + a1 b1, then fused + a2 b2. */
static float f32_fdot(const float *a, const float *b) {
    volatile float p = a[0] * b[0];
    return fmaf(a[2], b[2], fmaf(a[1], b[1], p));
}

static int f32_plane_ok(const float *n, const float *ax, float k2s) {
    float nv = f32_fdot(n, ax);
    if (nv >= 0.0f) return 1;
    float p[3] = {f32_fdot(n, ax + 3), f32_fdot(n, ax + 6), f32_fdot(n, ax + 9)};
    volatile float ss = f32_fdot(p, p);
    volatile float rhs = k2s * ss;
    volatile float lhs = nv * nv;
    return lhs <= rhs;
}

/* Half-tile mask of a (Gaussian, tile) pair whose cones overlap: bit 0 the
 * top half may be hit, bit 1 the bottom half; 0 = the tile is not reached. */
static unsigned f32_half_mask(const float *pl, const float *ax, float k2s, int inside) {
    const unsigned hb = pl[16] != 0.0f ? 2u : 0u;
    if (inside || pl[15] == 0.0f) return 1u | hb;
    if (!f32_plane_ok(pl + 6, ax, k2s) || !f32_plane_ok(pl + 9, ax, k2s)) return 0u;
    unsigned m = 0u;
    if (!hb) return f32_plane_ok(pl, ax, k2s) ? 1u : 0u;
    float nv = f32_fdot(pl + 12, ax);
    int mid_pos = 1, mid_neg = 1;   /* the ellipsoid reaches the top / bottom side of the mid plane */
    if (nv != 0.0f) {
        float p[3] = {f32_fdot(pl + 12, ax + 3), f32_fdot(pl + 12, ax + 6), f32_fdot(pl + 12, ax + 9)};
        volatile float ss = f32_fdot(p, p);
        volatile float rhs = k2s * ss;
        volatile float lhs = nv * nv;
        const int reach = lhs <= rhs;
        mid_pos = nv > 0.0f || reach;
        mid_neg = nv < 0.0f || reach;
    }
    if (mid_pos && f32_plane_ok(pl, ax, k2s)) m |= 1u;
    if (mid_neg && f32_plane_ok(pl + 3, ax, k2s)) m |= 2u;
    return m;
}

/* Light-space tile binning (Sec. 3.2, occluder culling), FP32 specification:
 * tiles of tile x tile texels, super-tiles of 8x8 tiles (on a cube map a
 * super-tile across two faces has one cone per face part, and overlapping
 * either counts); a Gaussian enters a
 * tile's list iff its bounding cone overlaps the super-tile's cone and the
 * tile's cone, and its culling ellipsoid reaches the tile's half-tile cones
 * (f32_half_mask; every Gaussian when the light is inside its bounding
 * sphere, and on tiles that straddle an octahedral face, both halves).
 * Writes pairs (key = l * n_tiles + tile, value = Gaussian index | half mask
 * << 30) in (key, Gaussian) order, up to `capacity`; returns the total number
 * of pairs (or -1 if an input was invalid). */
int64_t orc_f32_bin(const float *means, const float *scales, const float *quats, const float *opac,
                    int64_t N, const float *lights, int L, int H, int W, const float *radii, int K,
                    float kappa, float eps, int tile, uint32_t *keys, uint32_t *vals,
                    int64_t capacity) {
    int ty = (H + tile - 1) / tile, tx = (W + tile - 1) / tile;
    int sy = (ty + 7) / 8, sx = (tx + 7) / 8;
    int n_tiles = ty * tx;
    float *tc = (float *)malloc(sizeof(float) * 6 * n_tiles);
    float *tp = (float *)malloc(sizeof(float) * 17 * n_tiles);
    /* per super-tile: its cone, a second cone and a flag (1 when the
     * super-tile lies across two cube faces: one cone per face part) */
    float *sc = (float *)malloc(sizeof(float) * 13 * sy * sx);
    for (int a = 0; a < ty; ++a)
        for (int b = 0; b < tx; ++b) {
            int i0 = a * tile, j0 = b * tile;
            int i1 = i0 + tile < H ? i0 + tile : H, j1 = j0 + tile < W ? j0 + tile : W;
            orc_f32_rect_cone(i0, i1, j0, j1, H, W, tc + 6 * (a * tx + b));
            orc_f32_rect_planes(i0, i1, j0, j1, tile / 2, H, W, tp + 17 * (a * tx + b));
        }
    for (int a = 0; a < sy; ++a)
        for (int b = 0; b < sx; ++b) {
            int i0 = a * 8 * tile, j0 = b * 8 * tile;
            int i1 = i0 + 8 * tile < H ? i0 + 8 * tile : H, j1 = j0 + 8 * tile < W ? j0 + 8 * tile : W;
            float *sup = sc + 13 * (a * sx + b);
            sup[12] = 0.0f;
            if (g_atlas_map == 1 && (i1 - 1) / W == i0 / W + 1) {
                int cut = ((i1 - 1) / W) * W;
                orc_f32_rect_cone(i0, cut, j0, j1, H, W, sup);
                orc_f32_rect_cone(cut, i1, j0, j1, H, W, sup + 6);
                sup[12] = 1.0f;
            } else {
                orc_f32_rect_cone(i0, i1, j0, j1, H, W, sup);
            }
        }
    /* per tile: collect in Gaussian order (the natural (key, value) order) */
    int64_t total = 0;
    int bad = 0;
    float *cones = (float *)malloc(sizeof(float) * 9 * (N > 0 ? N : 1));
    float *axes = (float *)malloc(sizeof(float) * 12 * (N > 0 ? N : 1));
    float *k2s = (float *)malloc(sizeof(float) * (N > 0 ? N : 1));
    char *ok = (char *)malloc(N > 0 ? N : 1);
    for (int l = 0; l < L; ++l) {
        for (int64_t n = 0; n < N; ++n) {
            int r = orc_f32_gauss_cone(means + 3 * n, scales + 3 * n, opac[n], lights + 3 * l,
                                       kappa, eps, radii[K - 1], cones + 9 * n);
            for (int c = 0; c < 4; ++c)
                if (!isfinite(quats[4 * n + c])) r = -1;
            if (r < 0) bad = 1;
            ok[n] = r == 1;
            if (ok[n]) {
                orc_f32_gauss_axes(means + 3 * n, scales + 3 * n, quats + 4 * n, lights + 3 * l, axes + 12 * n);
                volatile float w = cones[9 * n + 6] * 1.0009765625f;
                k2s[n] = w;
            }
        }
        for (int t = 0; t < n_tiles; ++t) {
            int a = t / tx, b = t % tx;
            const float *sup = sc + 13 * ((a / 8) * sx + (b / 8));
            for (int64_t n = 0; n < N; ++n) {
                if (!ok[n]) continue;
                if (!f32_overlap(cones + 9 * n, sup) && !(sup[12] != 0.0f && f32_overlap(cones + 9 * n, sup + 6)))
                    continue;
                if (!f32_overlap(cones + 9 * n, tc + 6 * t)) continue;
                unsigned m = f32_half_mask(tp + 17 * t, axes + 12 * n, k2s[n], cones[9 * n + 5] != 0.0f);
                if (!m) continue;
                if (total < capacity) {
                    keys[total] = (uint32_t)(l * n_tiles + t);
                    vals[total] = (uint32_t)n | (m << 30);
                }
                ++total;
            }
        }
    }
    free(tc); free(tp); free(sc); free(cones); free(axes); free(k2s); free(ok);
    return bad ? -1 : total;
}

/* The same specification restricted to the listed (light, tile) keys
 * (key = l * n_tiles + tile, keys ascending): the pairs of those tiles only,
 * in (key, Gaussian) order, up to `capacity`; returns their total (or -1 if
 * an input was invalid).  Affordable at full size, where orc_f32_bin, which
 * tests every tile against every Gaussian, is not. */
int64_t orc_f32_bin_keys(const float *means, const float *scales, const float *quats, const float *opac,
                         int64_t N, const float *lights, int L, int H, int W, const float *radii, int K,
                         float kappa, float eps, int tile, const uint32_t *want, int n_want, uint32_t *keys,
                         uint32_t *vals, int64_t capacity) {
    int ty = (H + tile - 1) / tile, tx = (W + tile - 1) / tile;
    int n_tiles = ty * tx;
    int bad = 0;
    int64_t *cnt = (int64_t *)calloc((size_t)n_want + 1, sizeof(int64_t));
    float *cones = (float *)malloc(sizeof(float) * 9 * (N > 0 ? N : 1));
    float *axes = (float *)malloc(sizeof(float) * 12 * (N > 0 ? N : 1));
    float *k2s = (float *)malloc(sizeof(float) * (N > 0 ? N : 1));
    char *ok = (char *)malloc(N > 0 ? N : 1);
    int64_t written = 0;
    for (int l = 0; l < L; ++l) {
        int w0 = 0, w1 = 0;  /* the wanted keys of light l: [w0, w1) */
        while (w0 < n_want && (int)(want[w0] / n_tiles) < l) ++w0;
        w1 = w0;
        while (w1 < n_want && (int)(want[w1] / n_tiles) == l) ++w1;
        if (w1 == w0) continue;
        int bad_l = 0;
#pragma omp parallel for schedule(static) reduction(| : bad_l)
        for (int64_t n = 0; n < N; ++n) {
            int r = orc_f32_gauss_cone(means + 3 * n, scales + 3 * n, opac[n], lights + 3 * l, kappa, eps,
                                       radii[K - 1], cones + 9 * n);
            for (int c = 0; c < 4; ++c)
                if (!isfinite(quats[4 * n + c])) r = -1;
            if (r < 0) bad_l = 1;
            ok[n] = r == 1;
            if (ok[n]) {
                orc_f32_gauss_axes(means + 3 * n, scales + 3 * n, quats + 4 * n, lights + 3 * l, axes + 12 * n);
                volatile float w = cones[9 * n + 6] * 1.0009765625f;
                k2s[n] = w;
            }
        }
        bad |= bad_l;
        /* two passes over the wanted tiles: count, then write at the offsets */
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                int64_t acc = written;
                for (int q = w0; q < w1; ++q) {
                    int64_t c = cnt[q];
                    cnt[q] = acc;
                    acc += c;
                }
                written = acc;
            }
#pragma omp parallel for schedule(dynamic, 1)
            for (int q = w0; q < w1; ++q) {
                int t = (int)(want[q] % n_tiles);
                int a = t / tx, b = t % tx;
                int i0 = a * tile, j0 = b * tile;
                int i1 = i0 + tile < H ? i0 + tile : H, j1 = j0 + tile < W ? j0 + tile : W;
                int si0 = (a / 8) * 8 * tile, sj0 = (b / 8) * 8 * tile;
                int si1 = si0 + 8 * tile < H ? si0 + 8 * tile : H, sj1 = sj0 + 8 * tile < W ? sj0 + 8 * tile : W;
                float tc[6], tp[17], sup[13];
                orc_f32_rect_cone(i0, i1, j0, j1, H, W, tc);
                orc_f32_rect_planes(i0, i1, j0, j1, tile / 2, H, W, tp);
                sup[12] = 0.0f;
                if (g_atlas_map == 1 && (si1 - 1) / W == si0 / W + 1) {
                    int cut = ((si1 - 1) / W) * W;
                    orc_f32_rect_cone(si0, cut, sj0, sj1, H, W, sup);
                    orc_f32_rect_cone(cut, si1, sj0, sj1, H, W, sup + 6);
                    sup[12] = 1.0f;
                } else {
                    orc_f32_rect_cone(si0, si1, sj0, sj1, H, W, sup);
                }
                int64_t c = 0, pos = pass == 1 ? cnt[q] : 0;
                for (int64_t n = 0; n < N; ++n) {
                    if (!ok[n]) continue;
                    if (!f32_overlap(cones + 9 * n, sup) && !(sup[12] != 0.0f && f32_overlap(cones + 9 * n, sup + 6)))
                        continue;
                    if (!f32_overlap(cones + 9 * n, tc)) continue;
                    unsigned m = f32_half_mask(tp, axes + 12 * n, k2s[n], cones[9 * n + 5] != 0.0f);
                    if (!m) continue;
                    if (pass == 1 && pos < capacity) {
                        keys[pos] = want[q];
                        vals[pos] = (uint32_t)n | (m << 30);
                    }
                    ++pos;
                    ++c;
                }
                if (pass == 0) cnt[q] = c;
            }
        }
    }
    free(cnt); free(cones); free(axes); free(k2s); free(ok);
    return bad ? -1 : written;
}

/* Number of Gaussian-ray evaluations the method must make at the listed
 * texels (l,i,j): pairs whose ray from light l cuts the Gaussian's culling
 * ellipsoid {(x-mu)^T A (x-mu) <= k^2} at t > 0 (k^2 from the binning
 * specification).  m^2 = c - b^2/a and s* = -b/a in FP64.  This is the unit
 * count of the throughput metric. */
int64_t orc_count_ray_evals(const float *means, const float *scales, const float *quats,
                            const float *opac, int64_t N, const float *lights, int H, int W,
                            const float *radii, int K, float kappa, float eps,
                            const int32_t *lij, int64_t n_texels) {
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int64_t t = 0; t < n_texels; ++t) {
        int l = lij[3 * t], i = lij[3 * t + 1], j = lij[3 * t + 2];
        const float *o = lights + 3 * l;
        double od[3] = {o[0], o[1], o[2]}, d[3];
        orc_texel_dir(i, j, H, W, d);
        for (int64_t n = 0; n < N; ++n) {
            float cone[9];
            if (orc_f32_gauss_cone(means + 3 * n, scales + 3 * n, opac[n], o, kappa, eps,
                                   radii[K - 1], cone) != 1)
                continue;
            double A[9], a, b, c;
            orc_precision(scales + 3 * n, quats + 4 * n, A);
            double om[3] = {od[0] - means[3 * n], od[1] - means[3 * n + 1], od[2] - means[3 * n + 2]};
            orc_ray_coeffs(A, d, om, &a, &b, &c);
            double m2 = c - b * b / a;
            if (m2 <= (double)cone[6] && (cone[5] != 0.0f || -b / a > 0)) ++total;
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* HDRI probe (Sec. 3.4): real SH basis to degree 2 and the ridge fit, Eq. 7 */
/* ------------------------------------------------------------------------ */

/* Real SH basis Y_k, k = l^2 + l + m, degree <= 2, no Condon-Shortley phase:
 * Y_{1,-1} ~ y, Y_{1,0} ~ z, Y_{1,1} ~ x.  Constants from
 * Y_lm normalisation sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0). */
void orc_sh_basis(const double *d, double *Y) {
    double x = d[0], y = d[1], z = d[2];
    double c0 = 0.5 * sqrt(1.0 / ORC_PI);
    double c1 = sqrt(3.0 / (4.0 * ORC_PI));
    double c2 = 0.5 * sqrt(15.0 / ORC_PI);
    double c20 = 0.25 * sqrt(5.0 / ORC_PI);
    double c22 = 0.25 * sqrt(15.0 / ORC_PI);
    Y[0] = c0;
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
    Y[4] = c2 * x * y;
    Y[5] = c2 * y * z;
    Y[6] = c20 * (3.0 * z * z - 1.0);
    Y[7] = c2 * x * z;
    Y[8] = c22 * (x * x - y * y);
}

/* Eq. 7: (B^T W B + lambda I) A = B^T W Y, solved by Cholesky.  sh_out is
 * SH in R^{3 x 9}: sh_out[c*9 + k] = A[k][c].  Returns 0, or 1 if the system
 * is not positive definite. */
int orc_sh_fit(const float *dirs, const float *rgb, const float *w, int64_t n, double lambda,
               double *sh_out) {
    double G[81] = {0}, R[27] = {0};
    for (int64_t s = 0; s < n; ++s) {
        double d[3] = {dirs[3 * s], dirs[3 * s + 1], dirs[3 * s + 2]}, Y[9];
        orc_sh_basis(d, Y);
        double ws = w[s];
        for (int a = 0; a < 9; ++a) {
            for (int b = 0; b < 9; ++b) G[9 * a + b] += ws * Y[a] * Y[b];
            for (int c = 0; c < 3; ++c) R[3 * a + c] += ws * Y[a] * (double)rgb[3 * s + c];
        }
    }
    for (int a = 0; a < 9; ++a) G[9 * a + a] += lambda;
    /* Cholesky G = L L^T */
    double Lm[81] = {0};
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = G[9 * i + j];
            for (int k = 0; k < j; ++k) s -= Lm[9 * i + k] * Lm[9 * j + k];
            if (i == j) {
                if (!(s > 0)) return 1;
                Lm[9 * i + i] = sqrt(s);
            } else {
                Lm[9 * i + j] = s / Lm[9 * j + j];
            }
        }
    for (int c = 0; c < 3; ++c) {
        double yv[9], xv[9];
        for (int i = 0; i < 9; ++i) {
            double s = R[3 * i + c];
            for (int k = 0; k < i; ++k) s -= Lm[9 * i + k] * yv[k];
            yv[i] = s / Lm[9 * i + i];
        }
        for (int i = 8; i >= 0; --i) {
            double s = yv[i];
            for (int k = i + 1; k < 9; ++k) s -= Lm[9 * k + i] * xv[k];
            xv[i] = s / Lm[9 * i + i];
        }
        for (int k = 0; k < 9; ++k) sh_out[9 * c + k] = xv[k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Radiance transfer (Sec. 3.5, Eqs. 8-10)                                   */
/* ------------------------------------------------------------------------ */

/* Unit normal of a Gaussian: its smallest-scale axis (first one on ties),
 * flipped to point away from `centroid`. */
void orc_gauss_normal(const float *mu, const float *s, const float *q, const float *centroid,
                      double *n) {
    double R[9];
    orc_quat_to_rot(q, R);
    int k = 0;
    if (s[1] < s[k]) k = 1;
    if (s[2] < s[k]) k = 2;
    n[0] = R[0 + k]; n[1] = R[3 + k]; n[2] = R[6 + k];
    double side = n[0] * ((double)mu[0] - centroid[0]) + n[1] * ((double)mu[1] - centroid[1]) +
                  n[2] * ((double)mu[2] - centroid[2]);
    if (side < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
}

/* Eq. 10 for one normal: lat-long cell centres theta_i = (i+1/2) pi / n_theta,
 * phi_j = (j+1/2) 2 pi / n_phi, weights w = sin theta, L_c(omega) from Eq. 8,
 * S = max(0, <omega, n>)^q (Eq. 9). */
void orc_transfer_scale(const double *sh, const double *n, double q, double t_max, double eps,
                        int n_theta, int n_phi, double *s_out) {
    double num[3] = {0, 0, 0}, den = 0;
    for (int i = 0; i < n_theta; ++i) {
        double th = (i + 0.5) * ORC_PI / n_theta;
        for (int j = 0; j < n_phi; ++j) {
            double ph = (j + 0.5) * 2.0 * ORC_PI / n_phi;
            double om[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
            double wj = sin(th);
            double cs = om[0] * n[0] + om[1] * n[1] + om[2] * n[2];
            double S = cs > 0 ? pow(cs, q) : 0.0;
            double Y[9];
            orc_sh_basis(om, Y);
            for (int c = 0; c < 3; ++c) {
                double Lc = 0;
                for (int k = 0; k < 9; ++k) Lc += sh[9 * c + k] * Y[k];
                num[c] += wj * Lc * S;
            }
            den += wj * S;
        }
    }
    for (int c = 0; c < 3; ++c) {
        double v = num[c] / (den + eps);
        if (v < 0) v = 0;
        if (v > t_max) v = t_max;
        s_out[c] = v;
    }
}

/* Relit colours c' = max(0, gamma c (.) s(n)) for N Gaussians.  normals may
 * be NULL (then each normal is the smallest axis, away from centroid). */
void orc_relight(const double *sh, const float *means, const float *quats, const float *scales,
                 const float *normals, const float *centroid, const float *colors_in, int64_t N,
                 double q, double gamma, double t_max, double eps, int n_theta, int n_phi,
                 double *colors_out) {
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < N; ++g) {
        double n[3], s[3];
        if (normals) {
            double nn = sqrt((double)normals[3 * g] * normals[3 * g] +
                             (double)normals[3 * g + 1] * normals[3 * g + 1] +
                             (double)normals[3 * g + 2] * normals[3 * g + 2]);
            for (int c = 0; c < 3; ++c) n[c] = normals[3 * g + c] / nn;
        } else {
            orc_gauss_normal(means + 3 * g, scales + 3 * g, quats + 4 * g, centroid, n);
        }
        orc_transfer_scale(sh, n, q, t_max, eps, n_theta, n_phi, s);
        for (int c = 0; c < 3; ++c) {
            double v = gamma * (double)colors_in[3 * g + c] * s[c];
            colors_out[3 * g + c] = v > 0 ? v : 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Footprint sampling (Sec. 3.3 and ablation (A) of Sec. 4)                  */
/* ------------------------------------------------------------------------ */

/* Philox4x64-10, the counter-based generator of Salmon, Moraes, Dror and
 * Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds,
 * each taking the two 128-bit products M0 c0 and M1 c2 and mixing their
 * halves with c1, c3 and the round key; the key is advanced by the Weyl
 * constants between rounds. */
void orc_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0, p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normal number j of receiver q for seed `seed`: Philox4x64-10 at
 * counter (q, j / 8, 0, 0) and key (seed, 0) gives four 64-bit words; word
 * (j % 8) / 2 is split into two 32-bit halves, each giving a uniform
 * u = (h / 2^8 + 1) 2^-24 in (0, 1] from its top 24 bits; Box-Muller then
 * gives r cos(2 pi u2) for even j and r sin(2 pi u2) for odd j, with
 * r = sqrt(-2 ln u1). */
double orc_fp_normal(uint64_t seed, int64_t q, int j) {
    uint64_t ctr[4] = {(uint64_t)q, (uint64_t)(j / 8), 0, 0}, key[2] = {seed, 0}, w[4];
    orc_philox4x64(ctr, key, w);
    uint64_t word = w[(j % 8) / 2];
    uint32_t lo = (uint32_t)word, hi = (uint32_t)(word >> 32);
    double u1 = (double)((lo >> 8) + 1u) * (1.0 / 16777216.0);
    double u2 = (double)((hi >> 8) + 1u) * (1.0 / 16777216.0);
    double r = sqrt(-2.0 * log(u1));
    return (j % 2 == 0) ? r * cos(2.0 * ORC_PI * u2) : r * sin(2.0 * ORC_PI * u2);
}

/* Offsets z_i (n x 3) and weights w_i (sum 1) of one receiver's footprint.
 * mode 0: the centre alone (z = 0, w = 1).
 * mode 1: the 7-point stencil 0, +-e_x, +-e_y, +-e_z with weights proportional
 *         to exp(-|z|^2 / 2) (1 at the centre, e^-1/2 on the axes).
 * mode 2: n Monte Carlo offsets z_i ~ N(0, I) (orc_fp_normal, normal 3i + c
 *         for coordinate c), w_i = 1 / n.
 * Returns the number of samples. */
int orc_fp_offsets(int mode, int n_samples, uint64_t seed, int64_t q, double *z, double *w) {
    if (mode == 0) {
        z[0] = z[1] = z[2] = 0.0;
        w[0] = 1.0;
        return 1;
    }
    if (mode == 1) {
        double ea = exp(-0.5), norm = 1.0 + 6.0 * ea;
        for (int i = 0; i < 21; ++i) z[i] = 0.0;
        w[0] = 1.0 / norm;
        for (int a = 0; a < 3; ++a) {
            z[3 * (1 + 2 * a) + a] = 1.0;
            z[3 * (2 + 2 * a) + a] = -1.0;
            w[1 + 2 * a] = ea / norm;
            w[2 + 2 * a] = ea / norm;
        }
        return 7;
    }
    for (int i = 0; i < n_samples; ++i) {
        for (int c = 0; c < 3; ++c) z[3 * i + c] = orc_fp_normal(seed, q, 3 * i + c);
        w[i] = 1.0 / n_samples;
    }
    return n_samples;
}

/* Footprint attenuation: T_l = sum_i w_i T_l(x_i) with x_i = mu + R (s . z_i)
 * (rotation-aware offsets in the receiver's principal axes), then the direct
 * part of the colour is scaled as in orc_attenuate.  n_samples <= 64.
 * q_ids (may be NULL): the receiver index that keys the Monte Carlo offsets of
 * row q (default q), so a sample of receivers can be checked on its own. */
void orc_attenuate_footprint(const double *atlas, int L, int H, int W, const float *radii, int K,
                             const float *lights, const float *q_means, const float *q_quats,
                             const float *q_scales, const float *colors_in, int64_t Q,
                             const float *light_w, double direct_frac, int mode, int n_samples,
                             uint64_t seed, const int64_t *q_ids, double *colors_out,
                             double *T_out) {
    int64_t LS = (int64_t)K * H * W;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < Q; ++q) {
        double z[3 * 64], w[64], R[9];
        int n = orc_fp_offsets(mode, n_samples, seed, q_ids ? q_ids[q] : q, z, w);
        orc_quat_to_rot(q_quats + 4 * q, R);
        double pts[3 * 64];
        for (int i = 0; i < n; ++i)
            for (int r = 0; r < 3; ++r) {
                double acc = q_means[3 * q + r];
                for (int c = 0; c < 3; ++c) acc += R[3 * r + c] * ((double)q_scales[3 * q + c] * z[3 * i + c]);
                pts[3 * i + r] = acc;
            }
        double accl = 0;
        for (int l = 0; l < L; ++l) {
            double o[3] = {lights[3 * l], lights[3 * l + 1], lights[3 * l + 2]};
            double T = 0;
            for (int i = 0; i < n; ++i) T += w[i] * orc_sample_T(atlas + l * LS, H, W, radii, K, o, pts + 3 * i);
            if (T_out) T_out[q * L + l] = T;
            accl += (light_w ? (double)light_w[l] : 1.0 / L) * T;
        }
        double f = 1.0 - direct_frac + direct_frac * accl;
        for (int c = 0; c < 3; ++c) colors_out[3 * q + c] = (double)colors_in[3 * q + c] * f;
    }
}

/* ------------------------------------------------------------------------ */
/* Receiver-driven region of interest (Sec. 3.2)                             */
/* ------------------------------------------------------------------------ */

/* Receivers whose centres lie in the box B = {|x - c_x| <= R, |y - c_y| <= R,
 * z_min <= z <= z_max} (box = c_x, c_y, R, z_min, z_max; single-precision
 * decisions) mark, for each light, the texels their trilinear lookup reads:
 * the 2 x 2 bilinear taps of the FP32 index specification, clamped to the
 * edge (mask [L][H][W] of 0/1), and the shell range [k_min, k_max] of the two
 * shells bracketing their distance, clamped to [0, K-1] (krange [L][2];
 * k_min = K, k_max = -1 when no receiver sees the light).  A receiver at the
 * light reads nothing (T = 1 there). */
void orc_f32_roi(const float *recv, int64_t n, const float *box, const float *lights, int L, int H,
                 int W, const float *radii, int K, uint8_t *mask, int32_t *krange) {
    int64_t HW = (int64_t)H * W;
    memset(mask, 0, (size_t)(L * HW));
    for (int l = 0; l < L; ++l) {
        krange[2 * l] = K;
        krange[2 * l + 1] = -1;
    }
    for (int64_t q = 0; q < n; ++q) {
        const float *x = recv + 3 * q;
        volatile float dx = x[0] - box[0], dy = x[1] - box[1];
        if (!(fabsf(dx) <= box[2] && fabsf(dy) <= box[2] && x[2] >= box[3] && x[2] <= box[4])) continue;
        for (int l = 0; l < L; ++l) {
            int32_t oi[5];
            float of[3];
            orc_f32_sample_index(x, lights + 3 * l, H, W, radii, K, oi, of);
            if (of[2] == 0.0f) continue;
            int i0 = oi[2], j0 = oi[3], i1 = i0 + 1, j1 = j0 + 1;
            /* rows clamp to the point's face on a cube map, to the atlas otherwise */
            int rlo = 0, rhi = H - 1;
            if (g_atlas_map == 1) {
                rlo = (oi[0] / W) * W;
                rhi = rlo + W - 1;
            }
            i0 = i0 < rlo ? rlo : (i0 > rhi ? rhi : i0);
            i1 = i1 < rlo ? rlo : (i1 > rhi ? rhi : i1);
            j0 = j0 < 0 ? 0 : (j0 > W - 1 ? W - 1 : j0);
            j1 = j1 < 0 ? 0 : (j1 > W - 1 ? W - 1 : j1);
            uint8_t *m = mask + l * HW;
            m[(int64_t)i0 * W + j0] = m[(int64_t)i0 * W + j1] = 1;
            m[(int64_t)i1 * W + j0] = m[(int64_t)i1 * W + j1] = 1;
            int k = oi[4];
            int k0 = k < 0 ? 0 : (k > K - 1 ? K - 1 : k);
            int k1 = k < 0 ? 0 : (k + 1 > K - 1 ? K - 1 : k + 1);
            if (k0 < krange[2 * l]) krange[2 * l] = k0;
            if (k1 > krange[2 * l + 1]) krange[2 * l + 1] = k1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Cubemap probe render (Sec. 3.4): brute force over every Gaussian          */
/* ------------------------------------------------------------------------ */

/* Face f: forward axis F, texel axes U (columns u), V (rows v) as (axis, sign):
 * (+x, -z, -y), (-x, +z, -y), (+y, +x, +z), (-y, +x, -z), (+z, +x, -y), (-z, -x, -y). */
static const int kFaceAxis[6][3] = {{0, 2, 1}, {0, 2, 1}, {1, 0, 2}, {1, 0, 2}, {2, 0, 1}, {2, 0, 1}};
static const float kFaceSign[6][3] = {{1, -1, -1}, {-1, 1, -1}, {1, 1, 1}, {-1, 1, -1}, {1, 1, -1},
                                      {-1, -1, -1}};

typedef struct {
    float mx, my, A, B, C, tz;
    int ok;
} orc_splat;

/* R diag(s), single precision, each operation rounded on its own. */
static void f32_rot_scale(const float *q, const float *s, float *Rs) {
    float n = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    float w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[9] = {1.0f - 2.0f * (yy + zz), 2.0f * (xy - wz), 2.0f * (xz + wy),
                  2.0f * (xy + wz), 1.0f - 2.0f * (xx + zz), 2.0f * (yz - wx),
                  2.0f * (xz - wy), 2.0f * (yz + wx), 1.0f - 2.0f * (xx + yy)};
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Rs[3 * r + k] = R[3 * r + k] * s[k];
}

/* Dot product in a fixed order: (a0 b0 + a1 b1) + a2 b2, each step rounded. */
static float f32_dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
    float p0 = a0 * b0, p1 = a1 * b1, p2 = a2 * b2;
    return (p0 + p1) + p2;
}

/* The splat of a Gaussian in camera cam (16 floats: R row-major with rows x,
 * y, forward; position; fx, fy, cx, cy) for a W x H image: the mean's pixel
 * coordinates, the inverse of the screen covariance J W Sigma W^T J^T + 0.3 I
 * (J the Jacobian of the pinhole projection at the mean, its x/z and y/z
 * clamped to 1.3 x the half field of view) and the view depth.  Single
 * precision, each operation rounded on its own, in the kernel's order. */
static orc_splat f32_make_splat(const float *mu, const float *Rs, const float *cam, int W, int H,
                                float near) {
    orc_splat sp;
    memset(&sp, 0, sizeof(sp));
    const float *R = cam;
    float t0 = mu[0] - cam[9], t1 = mu[1] - cam[10], t2 = mu[2] - cam[11];
    float tx = f32_dot3(R[0], R[1], R[2], t0, t1, t2);
    float ty = f32_dot3(R[3], R[4], R[5], t0, t1, t2);
    float tz = f32_dot3(R[6], R[7], R[8], t0, t1, t2);
    sp.tz = tz;
    if (!(tz > near)) return sp;
    float fx = cam[12], fy = cam[13];
    float u = tx / tz, v = ty / tz;
    float fu = fx * u, fv = fy * v;
    sp.mx = fu + cam[14];
    sp.my = fv + cam[15];
    float gx[3], gy[3], gz[3], p1[3], p2[3];
    for (int k = 0; k < 3; ++k) {
        gx[k] = f32_dot3(R[0], R[1], R[2], Rs[k], Rs[3 + k], Rs[6 + k]);
        gy[k] = f32_dot3(R[3], R[4], R[5], Rs[k], Rs[3 + k], Rs[6 + k]);
        gz[k] = f32_dot3(R[6], R[7], R[8], Rs[k], Rs[3 + k], Rs[6 + k]);
    }
    float hw = 0.5f * (float)W, hh = 0.5f * (float)H;
    float qx = hw / fx, qy = hh / fy;
    float limx = 1.3f * qx, limy = 1.3f * qy;
    float uc = fminf(fmaxf(u, -limx), limx), vc = fminf(fmaxf(v, -limy), limy);
    for (int k = 0; k < 3; ++k) {
        float a1 = uc * gz[k], a2 = vc * gz[k];
        p1[k] = gx[k] - a1;
        p2[k] = gy[k] - a2;
    }
    float n11 = f32_dot3(p1[0], p1[1], p1[2], p1[0], p1[1], p1[2]);
    float n12 = f32_dot3(p1[0], p1[1], p1[2], p2[0], p2[1], p2[2]);
    float n22 = f32_dot3(p2[0], p2[1], p2[2], p2[0], p2[1], p2[2]);
    float hx = fx / tz, hy = fy / tz;
    float hxx = hx * hx, hxy = hx * hy, hyy = hy * hy;
    float a = hxx * n11 + 0.3f, b = hxy * n12, c = hyy * n22 + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return sp;
    sp.A = c / det;
    sp.B = -b / det;
    sp.C = a / det;
    sp.ok = 1;
    return sp;
}

static float f32_splat_m2(float px, float py, const orc_splat *sp) {
    float dx = px - sp->mx, dy = py - sp->my;
    float t1 = sp->A * (dx * dx), t2 = (2.0f * sp->B) * (dx * dy), t3 = sp->C * (dy * dy);
    return (t1 + t2) + t3;
}

typedef struct {
    uint32_t key;
    int64_t g;
    float m2;
} orc_hit;

static int hit_cmp(const void *x, const void *y) {
    const orc_hit *a = (const orc_hit *)x, *b = (const orc_hit *)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->g < b->g ? -1 : (a->g > b->g ? 1 : 0);
}

/* Radiance of pixels pix[0..npix) (index (v H + i) W + j) of n_views W x H
 * cameras (cams: n_views x 16 floats): every Gaussian with opacity > 0 whose
 * splat in view v covers the pixel centre within Mahalanobis distance 3
 * (single-precision decision), in order of depth (the float's bit pattern)
 * and then index, all composited front to back in double precision with
 * alpha = min(0.99, opacity exp(-m^2/2)), C += alpha T c, T *= 1 - alpha. */
void orc_render_view_pixels(const float *means, const float *scales, const float *quats, const float *opac,
                            const float *colors, int64_t n, const float *cams, int n_views, int W, int H,
                            float near, const int64_t *pix, int64_t npix, double *rgb_out) {
    orc_splat *sp = (orc_splat *)malloc(sizeof(orc_splat) * n_views * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        float Rs[9];
        f32_rot_scale(quats + 4 * g, scales + 3 * g, Rs);
        for (int v = 0; v < n_views; ++v)
            sp[(int64_t)n_views * g + v] = f32_make_splat(means + 3 * g, Rs, cams + 16 * v, W, H, near);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < npix; ++p) {
        int64_t q = pix[p];
        int v = (int)(q / ((int64_t)W * H));
        int rem = (int)(q - (int64_t)v * W * H), i = rem / W, j = rem - i * W;
        float px = (float)j + 0.5f, py = (float)i + 0.5f;
        size_t cap = 64, cnt = 0;
        orc_hit *hits = (orc_hit *)malloc(sizeof(orc_hit) * cap);
        for (int64_t g = 0; g < n; ++g) {
            const orc_splat *s = sp + (int64_t)n_views * g + v;
            if (!s->ok || !(opac[g] > 0.0f)) continue;
            float m2 = f32_splat_m2(px, py, s);
            if (!(m2 <= 9.0f)) continue;
            if (cnt == cap) {
                cap *= 2;
                hits = (orc_hit *)realloc(hits, sizeof(orc_hit) * cap);
            }
            uint32_t key;
            memcpy(&key, &s->tz, 4);
            hits[cnt].key = key;
            hits[cnt].g = g;
            hits[cnt].m2 = m2;
            ++cnt;
        }
        qsort(hits, cnt, sizeof(orc_hit), hit_cmp);
        double T = 1.0, c[3] = {0, 0, 0};
        for (size_t k = 0; k < cnt; ++k) {
            int64_t g = hits[k].g;
            double alpha = (double)opac[g] * exp(-0.5 * (double)hits[k].m2);
            if (alpha > 0.99) alpha = 0.99;
            for (int ch = 0; ch < 3; ++ch) c[ch] += alpha * T * (double)colors[3 * g + ch];
            T *= 1.0 - alpha;
        }
        for (int ch = 0; ch < 3; ++ch) rgb_out[3 * p + ch] = c[ch];
        free(hits);
    }
    free(sp);
}

/* The six probe cameras at `centre` (cams: 6 x 16 floats): rows U, V, F of
 * each face, fx = fy = cx = cy = face / 2. */
void orc_cube_cams(const float *centre, int face, float *cams) {
    for (int f = 0; f < 6; ++f) {
        float *c = cams + 16 * f;
        for (int k = 0; k < 9; ++k) c[k] = 0.0f;
        c[0 + kFaceAxis[f][1]] = kFaceSign[f][1];
        c[3 + kFaceAxis[f][2]] = kFaceSign[f][2];
        c[6 + kFaceAxis[f][0]] = kFaceSign[f][0];
        c[9] = centre[0];
        c[10] = centre[1];
        c[11] = centre[2];
        c[12] = c[13] = c[14] = c[15] = 0.5f * (float)face;
    }
}

/* Probe pixels (index f face^2 + i face + j) of the cube at `centre`. */
void orc_render_pixels(const float *means, const float *scales, const float *quats, const float *opac,
                       const float *colors, int64_t n, const float *centre, int face, float near,
                       const int64_t *pix, int64_t npix, double *rgb_out) {
    float cams[6 * 16];
    orc_cube_cams(centre, face, cams);
    orc_render_view_pixels(means, scales, quats, opac, colors, n, cams, 6, face, face, near, pix, npix, rgb_out);
}
