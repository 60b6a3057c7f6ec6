/*
 * mppi.c -- sampling, softmax update, shift and one MPPI step (oracle).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * arXiv 2409.10469, Sec. II-B:
 *   Gaussian samples u ~ N(mu, Sigma) around the mean (Alg. 1, sampling step),
 *   weights omega_n = exp(-(L_n - L_min)/lambda) / sum (Eq. 1),
 *   mean update mu = sum omega_n u_n (Eq. 2),
 *   apply u = mu[0], then mu <- shifted(mu) (Alg. 1, last three steps).
 * Sampling is over the 4 spline knots of 12 joint targets (Sec. III-B).
 *
 * Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Box-Muller
 * transform, in an FP32 operation sequence fixed by the model spec.  The ln and
 * sin/cos routines are the project's own: ln by exponent/mantissa split with
 * Cody-Waite ln2 (Cody & Waite 1980) and the atanh series
 * ln m = 2 (s + s^3/3 + s^5/5 + ...), s = (m-1)/(m+1); sin/cos by exact
 * quarter-turn reduction of a 24-bit fixed-point angle and Taylor polynomials.
 * This file is compiled with -ffp-contract=off; every fused step is an
 * explicit fmaf.
 */
#include <math.h>
#include <string.h>
#include <stdlib.h>
#include "oracle.h"

/* ---------------- Philox4x32-10 ---------------- */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------- FP32 ln and sincos (project-written) ---------------- */

static float f_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* natural log of a positive normal float */
float or_lnf(float x) {
    const float LN2_HI = 0.693145751953125f;        /* 0x3f317200: 16 significant bits */
    const float LN2_LO = 1.428606765e-06f;          /* 0x35bfbe8e: (float)(ln2 - LN2_HI) */
    const float SQRT2 = 1.41421354f;                /* 0x3fb504f3 */
    uint32_t b = bits_from_f(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = f_from_bits((b & 0x007fffffu) | 0x3f800000u);   /* [1, 2) */
    if (m > SQRT2) { m = m * 0.5f; e = e + 1; }                 /* [sqrt(1/2), sqrt(2)] */
    float f = m - 1.0f;                                         /* exact */
    float s = f / (m + 1.0f);
    float z = s * s;
    float p = fmaf(z, 1.0f / 9.0f, 1.0f / 7.0f);
    p = fmaf(z, p, 1.0f / 5.0f);
    p = fmaf(z, p, 1.0f / 3.0f);
    p = p * z;
    float s2 = s + s;                                           /* exact */
    float r = fmaf(s2, p, s2);                                  /* 2 atanh(s) */
    float ef = (float)e;
    return fmaf(ef, LN2_HI, fmaf(ef, LN2_LO, r));
}

/* cos and sin of 2 pi n / 2^24 for a 24-bit integer n */
void or_sincos2pi_u24(uint32_t n, float* c, float* s) {
    const float HALF_PI = 1.57079637f;                          /* 0x3fc90fdb */
    const float S3 = -1.0f / 6.0f, S5 = 1.0f / 120.0f, S7 = -1.0f / 5040.0f, S9 = 1.0f / 362880.0f;
    const float C2 = -0.5f, C4 = 1.0f / 24.0f, C6 = -1.0f / 720.0f, C8 = 1.0f / 40320.0f,
                C10 = -1.0f / 3628800.0f;
    uint32_t qd = (n >> 22) & 3u;
    int32_t fr = (int32_t)(n & 0x3fffffu);
    if (fr >= 0x200000) { fr -= 0x400000; qd = (qd + 1u) & 3u; }
    float t = (float)fr * (1.0f / 4194304.0f);                  /* exact, [-1/2, 1/2) */
    float xr = t * HALF_PI;                                     /* [-pi/4, pi/4) */
    float x2 = xr * xr;
    float ps = fmaf(x2, S9, S7);
    ps = fmaf(x2, ps, S5);
    ps = fmaf(x2, ps, S3);
    float sn = fmaf(xr * x2, ps, xr);
    float pc = fmaf(x2, C10, C8);
    pc = fmaf(x2, pc, C6);
    pc = fmaf(x2, pc, C4);
    pc = fmaf(x2, pc, C2);
    float cs = fmaf(x2, pc, 1.0f);
    switch (qd) {
        case 0: *c = cs;  *s = sn;  break;
        case 1: *c = -sn; *s = cs;  break;
        case 2: *c = -cs; *s = -sn; break;
        default: *c = sn; *s = -cs; break;
    }
}

/* two N(0,1) draws from two uint32: u1 = (a>>8 + 1) 2^-24 in (0,1], angle 2 pi (b>>8) 2^-24 */
void or_box_muller(uint32_t a, uint32_t b, float* e0, float* e1) {
    float u1 = (float)((a >> 8) + 1u) * (1.0f / 16777216.0f);
    float l = or_lnf(u1);
    float r = sqrtf(-2.0f * l);
    float c, s;
    or_sincos2pi_u24(b >> 8, &c, &s);
    *e0 = r * c;
    *e1 = r * s;
}

/* the first D normals (D a multiple of 4) of sample k: Philox calls g = 0 .. D/4 - 1,
 * counter (g, k, step, inst), key = seed; 48 normals for the knot representations */
static void noise_dim(uint64_t seed, uint32_t step, uint32_t inst, uint32_t k, int D, float* eps) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t g = 0; g < (uint32_t)(D / 4); g++) {
        uint32_t ctr[4] = {g, k, step, inst}, r[4];
        or_philox4x32_10(ctr, key, r);
        or_box_muller(r[0], r[1], &eps[4 * g + 0], &eps[4 * g + 1]);
        or_box_muller(r[2], r[3], &eps[4 * g + 2], &eps[4 * g + 3]);
    }
}

void or_noise(uint64_t seed, uint32_t step, uint32_t inst, uint32_t k, float eps[OR_D]) {
    noise_dim(seed, step, inst, k, OR_D, eps);
}

/*
 * Samples U[K][D], D = or_param_dim(interp, H): knots [knot][joint] (D = 48) or
 * direct targets [t][joint] (D = 12 H, sigma of joint i = sigma[i], the first
 * knot's).  Sample 0 is the nominal mean; when n_prop > 0 the last n_prop
 * samples are drawn around mu_prop and the first of them is mu_prop itself.
 * U = clamp(fmaf(sigma, eps, centre), lo, hi).
 */
void or_sample(const or_mppi* m, const float* mu, const float* mu_prop, uint32_t step,
               float* U) {
    const int D = or_param_dim(m->interp, m->H);
    int kp0 = m->K - (mu_prop ? m->n_prop : 0);
    float* eps = (float*)malloc(sizeof(float) * (size_t)D);
    for (int k = 0; k < m->K; k++) {
        const float* ctrv = (k >= kp0) ? mu_prop : mu;
        int nominal = (k == 0) || (k == kp0 && mu_prop);
        if (nominal) memset(eps, 0, sizeof(float) * (size_t)D);
        else noise_dim(m->seed, step, m->inst, (uint32_t)k, D, eps);
        for (int d = 0; d < D; d++) {
            int jt = d % 3;
            float c = ctrv[d];
            if (k >= kp0 && !isfinite(c)) c = mu[d];   /* non-finite proposal: the plain mean */
            float sg = m->interp == OR_INTERP_DIRECT ? m->sigma[d % OR_NJ] : m->sigma[d];
            float v = fmaf(sg, eps[d], c);
            v = fmaxf(v, m->q_lo[jt]);
            v = fminf(v, m->q_hi[jt]);
            U[(size_t)k * D + d] = v;
        }
    }
    free(eps);
}

/* ---------------- Eq. 1, Eq. 2 ---------------- */

/*
 * Softmax weights over finite costs and the weighted mean of the knots.
 * Returns 0, or -1 when no cost is finite (mu_out left untouched).
 */
int or_update_dim(const double* L, const float* U, int K, int D, double lambda, float* mu_out,
                  double* w_out) {
    double Lmin = INFINITY;
    for (int k = 0; k < K; k++)
        if (isfinite(L[k]) && L[k] < Lmin) Lmin = L[k];
    if (!isfinite(Lmin)) return -1;
    double* w = w_out ? w_out : (double*)malloc(sizeof(double) * K);
    double Z = 0;
    for (int k = 0; k < K; k++) {
        w[k] = isfinite(L[k]) ? exp(-(L[k] - Lmin) / lambda) : 0.0;
        Z += w[k];
    }
    for (int k = 0; k < K; k++) w[k] /= Z;
    for (int d = 0; d < D; d++) {
        double s = 0;
        for (int k = 0; k < K; k++) s += w[k] * (double)U[(size_t)k * D + d];
        mu_out[d] = (float)s;
    }
    if (!w_out) free(w);
    return 0;
}

int or_update_d(const double* L, const float* U, int K, double lambda, float mu_out[OR_D],
                double* w_out) {
    return or_update_dim(L, U, K, OR_D, lambda, mu_out, w_out);
}

int or_update(const float* L, const float* U, int K, double lambda, float mu_out[OR_D],
              double* w_out) {
    double* Ld = (double*)malloc(sizeof(double) * (K > 0 ? K : 1));
    for (int k = 0; k < K; k++) Ld[k] = (double)L[k];
    int r = or_update_d(Ld, U, K, lambda, mu_out, w_out);
    free(Ld);
    return r;
}

/*
 * shifted(mu): re-sample the knot spline at tau_j + delta, delta = one control
 * period in normalised time, ctrl_steps / (H - 1); times past the end are held
 * at tau = 1.
 */
void or_shift(const float mu[OR_D], int H, int ctrl_steps, float mu_out[OR_D]) {
    double delta = (H > 1) ? (double)ctrl_steps / (double)(H - 1) : 0.0;
    float tmp[OR_D];
    for (int j = 0; j < OR_NKNOT; j++) {
        real u[OR_NJ];
        or_spline_eval(mu, j / 3.0 + delta, u);
        for (int i = 0; i < OR_NJ; i++) tmp[j * OR_NJ + i] = (float)u[i];
    }
    memcpy(mu_out, tmp, sizeof(tmp));
}

/*
 * shifted(mu) for any representation: the knot representations re-sample their
 * own interpolant at tau_j + delta (held at tau = 1 past the end); direct
 * targets move ctrl_steps steps earlier, the last one held.
 */
void or_shift_mode(const float* mu, int interp, int H, int ctrl_steps, float* mu_out) {
    if (interp == OR_INTERP_CUBIC) {
        or_shift(mu, H, ctrl_steps, mu_out);
        return;
    }
    if (interp == OR_INTERP_DIRECT) {
        float* tmp = (float*)malloc(sizeof(float) * (size_t)OR_NJ * H);
        for (int t = 0; t < H; t++) {
            int src = t + ctrl_steps < H ? t + ctrl_steps : H - 1;
            for (int i = 0; i < OR_NJ; i++) tmp[t * OR_NJ + i] = mu[src * OR_NJ + i];
        }
        memcpy(mu_out, tmp, sizeof(float) * (size_t)OR_NJ * H);
        free(tmp);
        return;
    }
    /* zeroth / linear: the interpolant at 3 tau = j + 3 ctrl_steps / (H - 1), held at 3;
     * its integer part and fraction from integer arithmetic */
    float tmp[OR_D];
    const int den = H > 1 ? H - 1 : 1, num = H > 1 ? 3 * ctrl_steps : 0;
    for (int j = 0; j < OR_NKNOT; j++) {
        int jj = j + num / den;
        double f = (double)(num % den) / (double)den;
        if (jj >= 3) { jj = 3; f = 0; }
        for (int i = 0; i < OR_NJ; i++) {
            double v;
            if (interp == OR_INTERP_ZERO) {
                v = mu[jj * OR_NJ + i];
            } else if (jj == 3) {
                v = mu[3 * OR_NJ + i];
            } else {
                v = (1 - f) * mu[jj * OR_NJ + i] + f * mu[(jj + 1) * OR_NJ + i];
            }
            tmp[j * OR_NJ + i] = (float)v;
        }
    }
    memcpy(mu_out, tmp, sizeof(tmp));
}

/*
 * One control step of Alg. 1: sample, roll out from x0, weight (Eq. 1),
 * update (Eq. 2), take u0 = the controls of step 0 (knot 0 for every knot
 * representation, the first direct target otherwise), shift.  mu (D floats) is
 * updated in place.  L_out (float costs) and U_out are optional.
 * Returns 0, or -1 when every cost is non-finite (mu kept, u0 = mu[0]).
 */
int or_mppi_step(const or_world* w, const or_cost* c, const or_mppi* m, const double* x0,
                 float* mu, const float* mu_prop, uint32_t step, float u0[OR_NJ],
                 float* L_out, float* U_out, int nthreads) {
    int K = m->K;
    const int D = or_param_dim(m->interp, m->H);
    float* U = U_out ? U_out : (float*)malloc(sizeof(float) * (size_t)K * D);
    double* L = (double*)malloc(sizeof(double) * K);
    or_sample(m, mu, mu_prop, step, U);
    double t0 = (double)step * m->ctrl_steps * m->dt;
    or_rollouts(w, c, m, t0, x0, 0, U, K, L, NULL, nthreads);
    if (L_out)
        for (int k = 0; k < K; k++) L_out[k] = (float)L[k];
    float* mnew = (float*)malloc(sizeof(float) * (size_t)D);
    int rc = or_update_dim(L, U, K, D, m->lambda, mnew, NULL);
    if (rc != 0) memcpy(mnew, mu, sizeof(float) * (size_t)D);
    for (int j = 0; j < OR_NJ; j++) u0[j] = mnew[j];
    or_shift_mode(mnew, m->interp, m->H, m->ctrl_steps, mu);
    free(mnew);
    free(L);
    if (!U_out) free(U);
    return rc;
}

/* ---------------- helpers for the Python test harness ---------------- */

size_t or_world_size(void) { return sizeof(or_world); }
size_t or_tree_size(void) { return sizeof(or_tree); }

void or_lnf_many(const float* x, float* y, long n) {
    for (long i = 0; i < n; i++) y[i] = or_lnf(x[i]);
}

void or_sincos_u24_many(const uint32_t* nn, float* c, float* s, long n) {
    for (long i = 0; i < n; i++) or_sincos2pi_u24(nn[i] & 0xffffffu, &c[i], &s[i]);
}

void or_noise_many(uint64_t seed, uint32_t step, uint32_t inst, const uint32_t* ks, long n,
                   float* eps) {
    for (long i = 0; i < n; i++) or_noise(seed, step, inst, ks[i], eps + (size_t)i * OR_D);
}
