/*
 * Differentiable form of the render path, binary64 (TEST INFRASTRUCTURE ONLY:
 * see oracle.h; shares nothing with the CUDA library).
 *
 * Per-Gaussian parameters follow the 3D Gaussian splatting parametrisation the
 * paper builds on (§3.1): mean mu, log-scale s, quaternion q = (w, x, y, z) of
 * any non-zero norm, opacity logit l and SH coefficients c_k:
 *   Sigma   = R(q/|q|) diag(e^{2 s}) R(q/|q|)^T
 *   alpha0  = 1 / (1 + e^{-l}),  l clamped to [-80, 80]
 *   colour  = max(0, 1/2 + sum_k Y_k(d) c_k),  d = (mu - campos) / |mu - campos|
 * and the screen-space Gaussian of Eq. 1 is the EWA splat of oracle.c (J W Sigma
 * W^T J^T + 0.3 I, its inverse the conic), blended by Eq. 2.
 *
 * The selection (the LoD cut of §3.2), the pair lists and every skip / stop /
 * clamp decision of blending are discrete; the gradient is the one of the
 * smooth function obtained by freezing them (a fixed cut, as when the cut is
 * trained).  oracle_trace_pixels (oracle.c) records them per pixel from the
 * binary32 decision path; the functions below evaluate and differentiate the
 * frozen function in binary64:
 *   C(p) = sum_i c_i alpha_i T_i + bg T_{K+1},  T_1 = 1,  T_{i+1} = T_i (1 - alpha_i),
 *   alpha_i = 0.99 for a recorded clamp, else alpha0_i exp(power_i(p)).
 *
 * oracle_prep_params computes the binary32 attributes the decisions are taken
 * on (Sigma, alpha0, ln alpha0) from the parameters in one fixed operation
 * order, so that any IEEE binary32 implementation of the same order returns the
 * same bits.
 *
 * Must be compiled with -ffp-contract=off and without -ffast-math.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LOGIT_MAX 80.0f
#define LOWPASS64 0.3
#define GUARD64 1.3

/* ------------------------------------------------------------------ */
/* binary32 parameter -> attribute map                                */
/* ------------------------------------------------------------------ */

/* ln x for positive normal binary32 x.  x = 2^e m with m in [sqrt(1/2), sqrt(2)]
 * (exponent bits), ln m = 2 atanh(s) with s = (m - 1) / (m + 1), |s| < 0.172,
 * summed as the odd series 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9) by Horner's
 * rule (truncation below 1e-9 relative; Abramowitz & Stegun 4.1.27), plus
 * e ln 2.  Fixed order, no fused operations. */
float oracle_lnf(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xffu) - 127;
    const uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 1.41421356f) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float p = 0.111111111f;
    p = p * s2 + 0.142857143f;
    p = p * s2 + 0.2f;
    p = p * s2 + 0.333333333f;
    p = p * s2 + 1.0f;
    const float lm = (2.0f * s) * p;
    return (float)e * 0.693147182f + lm;
}

void oracle_prep_params(int32_t n, const float* log_scale, const float* quat, const float* logit,
                        float* cov_out, float* opacity_out, float* ln_opacity_out)
{
    for (int32_t i = 0; i < n; ++i) {
        float w = quat[i], x = quat[n + i], y = quat[2 * n + i], z = quat[3 * n + i];
        const float qn = sqrtf(((w * w + x * x) + y * y) + z * z);
        w = w / qn;
        x = x / qn;
        y = y / qn;
        z = z / qn;
        float R[3][3];
        R[0][0] = 1.0f - 2.0f * (y * y + z * z);
        R[0][1] = 2.0f * (x * y - w * z);
        R[0][2] = 2.0f * (x * z + w * y);
        R[1][0] = 2.0f * (x * y + w * z);
        R[1][1] = 1.0f - 2.0f * (x * x + z * z);
        R[1][2] = 2.0f * (y * z - w * x);
        R[2][0] = 2.0f * (x * z - w * y);
        R[2][1] = 2.0f * (y * z + w * x);
        R[2][2] = 1.0f - 2.0f * (x * x + y * y);
        float s2[3];
        for (int k = 0; k < 3; ++k) s2[k] = oracle_expf(2.0f * log_scale[k * n + i]);
        static const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        for (int e = 0; e < 6; ++e) {
            const int a = ij[e][0], c = ij[e][1];
            cov_out[e * n + i] = ((R[a][0] * s2[0]) * R[c][0] + (R[a][1] * s2[1]) * R[c][1]) +
                                 (R[a][2] * s2[2]) * R[c][2];
        }
        float l = logit[i];
        l = l < -LOGIT_MAX ? -LOGIT_MAX : (l > LOGIT_MAX ? LOGIT_MAX : l);
        const float den = 1.0f + oracle_expf(-l);
        opacity_out[i] = 1.0f / den;
        ln_opacity_out[i] = -oracle_lnf(den);
    }
}

/* ------------------------------------------------------------------ */
/* binary64 forward of one Gaussian                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    double W[3][3], t[3];        /* camera */
    double fx, fy, cx, cy, limx, limy, campos[3];
} cam64;

static cam64 to_cam64(const ocam* c)
{
    cam64 k;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) k.W[i][j] = c->R[3 * i + j];
        k.t[i] = c->t[i];
        k.campos[i] = c->campos[i];
    }
    k.fx = c->fx;
    k.fy = c->fy;
    k.cx = c->cx;
    k.cy = c->cy;
    k.limx = GUARD64 * (double)c->tan_half_x;
    k.limy = GUARD64 * (double)c->tan_half_y;
    return k;
}

typedef struct {
    /* outputs */
    double u, v, A, B, C, a0, rgb[3];
    /* intermediates for the backward */
    double p[3];                 /* camera-space centre */
    int clx, cly;                /* tangent clamped (0 inside the guard band) */
    double tx, ty;               /* clamped tangents times depth */
    double J[2][3], M[2][3], S[3][3], R[3][3], s2[3], qh[4], qn;
    double a, b, c, det;
    double dir[3], dlen, Y[16], pre[3];
    double l;
    int l_clamped;
} gfwd;

static void rot_of(const double q[4], double R[3][3])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void forward_gauss(const cam64* k, const oparams64* P, int64_t n, gfwd* g)
{
    const int64_t N = P->n;
    const int K = (P->sh_degree + 1) * (P->sh_degree + 1);
    double mu[3] = {P->mu[n], P->mu[N + n], P->mu[2 * N + n]};
    /* Sigma */
    double q[4];
    for (int i = 0; i < 4; ++i) q[i] = P->quat[i * N + n];
    g->qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) g->qh[i] = q[i] / g->qn;
    rot_of(g->qh, g->R);
    for (int i = 0; i < 3; ++i) g->s2[i] = exp(2.0 * P->log_scale[i * N + n]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int m = 0; m < 3; ++m) v += g->R[i][m] * g->s2[m] * g->R[j][m];
            g->S[i][j] = v;
        }
    /* camera space and EWA Jacobian */
    for (int i = 0; i < 3; ++i)
        g->p[i] = k->W[i][0] * mu[0] + k->W[i][1] * mu[1] + k->W[i][2] * mu[2] + k->t[i];
    const double z = g->p[2];
    double rx = g->p[0] / z, ry = g->p[1] / z;
    g->clx = rx < -k->limx ? -1 : (rx > k->limx ? 1 : 0);
    g->cly = ry < -k->limy ? -1 : (ry > k->limy ? 1 : 0);
    if (g->clx) rx = g->clx * k->limx;
    if (g->cly) ry = g->cly * k->limy;
    g->tx = rx * z;
    g->ty = ry * z;
    g->J[0][0] = k->fx / z;
    g->J[0][1] = 0.0;
    g->J[0][2] = -k->fx * g->tx / (z * z);
    g->J[1][0] = 0.0;
    g->J[1][1] = k->fy / z;
    g->J[1][2] = -k->fy * g->ty / (z * z);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            g->M[i][j] = g->J[i][0] * k->W[0][j] + g->J[i][1] * k->W[1][j] + g->J[i][2] * k->W[2][j];
    double S2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double v = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) v += g->M[i][a] * g->S[a][b] * g->M[j][b];
            S2[i][j] = v;
        }
    g->a = S2[0][0] + LOWPASS64;
    g->b = S2[0][1];
    g->c = S2[1][1] + LOWPASS64;
    g->det = g->a * g->c - g->b * g->b;
    g->A = g->c / g->det;
    g->B = -g->b / g->det;
    g->C = g->a / g->det;
    g->u = k->fx * g->p[0] / z + k->cx;
    g->v = k->fy * g->p[1] / z + k->cy;
    /* opacity */
    double l = P->logit[n];
    g->l_clamped = l < -LOGIT_MAX || l > LOGIT_MAX;
    if (l < -LOGIT_MAX) l = -LOGIT_MAX;
    if (l > LOGIT_MAX) l = LOGIT_MAX;
    g->l = l;
    g->a0 = 1.0 / (1.0 + exp(-l));
    /* view-dependent colour */
    for (int i = 0; i < 3; ++i) g->dir[i] = mu[i] - k->campos[i];
    g->dlen = sqrt(g->dir[0] * g->dir[0] + g->dir[1] * g->dir[1] + g->dir[2] * g->dir[2]);
    for (int i = 0; i < 3; ++i) g->dir[i] /= g->dlen;
    oracle_sh_basis(P->sh_degree, g->dir, g->Y);
    const double* c = P->sh + (size_t)n * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double v = 0.5;
        for (int kk = 0; kk < K; ++kk) v += g->Y[kk] * c[3 * kk + ch];
        g->pre[ch] = v;
        g->rgb[ch] = v > 0.0 ? v : 0.0;
    }
}

/* Partial derivatives of the Cartesian SH polynomials of oracle_sh_basis with
 * respect to (x, y, z), treating the three as independent. */
static void sh_basis_jac(int deg, const double d[3], double J[16][3])
{
    const double pi = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    memset(J, 0, sizeof(double) * 16 * 3);
    if (deg < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    J[1][1] = -k1;
    J[2][2] = k1;
    J[3][0] = -k1;
    if (deg < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    J[4][0] = k2a * y;          J[4][1] = k2a * x;
    J[5][1] = -k2a * z;         J[5][2] = -k2a * y;
    J[6][0] = -2.0 * k2b * x;   J[6][1] = -2.0 * k2b * y;   J[6][2] = 4.0 * k2b * z;
    J[7][0] = -k2a * z;         J[7][2] = -k2a * x;
    J[8][0] = 2.0 * k2c * x;    J[8][1] = -2.0 * k2c * y;
    if (deg < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    /* Y9 = -k3a (3 x^2 y - y^3) */
    J[9][0] = -k3a * 6.0 * x * y;
    J[9][1] = -k3a * (3.0 * x * x - 3.0 * y * y);
    /* Y10 = k3b x y z */
    J[10][0] = k3b * y * z;
    J[10][1] = k3b * x * z;
    J[10][2] = k3b * x * y;
    /* Y11 = -k3c (4 y z^2 - x^2 y - y^3) */
    J[11][0] = -k3c * (-2.0 * x * y);
    J[11][1] = -k3c * (4.0 * z * z - x * x - 3.0 * y * y);
    J[11][2] = -k3c * (8.0 * y * z);
    /* Y12 = k3d (2 z^3 - 3 x^2 z - 3 y^2 z) */
    J[12][0] = k3d * (-6.0 * x * z);
    J[12][1] = k3d * (-6.0 * y * z);
    J[12][2] = k3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    /* Y13 = -k3c (4 x z^2 - x^3 - x y^2) */
    J[13][0] = -k3c * (4.0 * z * z - 3.0 * x * x - y * y);
    J[13][1] = -k3c * (-2.0 * x * y);
    J[13][2] = -k3c * (8.0 * x * z);
    /* Y14 = k3e (x^2 z - y^2 z) */
    J[14][0] = k3e * 2.0 * x * z;
    J[14][1] = -k3e * 2.0 * y * z;
    J[14][2] = k3e * (x * x - y * y);
    /* Y15 = -k3a (x^3 - 3 x y^2) */
    J[15][0] = -k3a * (3.0 * x * x - 3.0 * y * y);
    J[15][1] = -k3a * (-6.0 * x * y);
}

/* ------------------------------------------------------------------ */
/* frozen blending                                                    */
/* ------------------------------------------------------------------ */

static int prepare(const ocam* c, const oparams64* P, const uint32_t* sel, int32_t M, cam64* k,
                   gfwd** out)
{
    *k = to_cam64(c);
    gfwd* g = (gfwd*)calloc((size_t)(M > 0 ? M : 1), sizeof(gfwd));
    if (!g) return -1;
    for (int32_t m = 0; m < M; ++m) forward_gauss(k, P, sel[m], &g[m]);
    *out = g;
    return 0;
}

static double alpha_of(const gfwd* g, int clamped, double px, double py, double* ex,
                       double* dx, double* dy)
{
    *dx = g->u - px;
    *dy = g->v - py;
    const double power = -0.5 * (g->A * *dx * *dx + g->C * *dy * *dy) - g->B * *dx * *dy;
    *ex = exp(power);
    return clamped ? 0.99 : g->a0 * *ex;
}

int oracle_diff_render(const ocam* c, const double bg[3], const oparams64* P, const uint32_t* sel,
                       int32_t M, const int64_t* pix, int64_t n_pix, const int64_t* offs,
                       const uint32_t* ent, double* rgb_out)
{
    cam64 k;
    gfwd* g;
    if (prepare(c, P, sel, M, &k, &g)) return -1;
    for (int64_t i = 0; i < n_pix; ++i) {
        const double px = (double)(pix[i] % c->width) + 0.5, py = (double)(pix[i] / c->width) + 0.5;
        double T = 1.0, acc[3] = {0.0, 0.0, 0.0};
        for (int64_t q = offs[i]; q < offs[i + 1]; ++q) {
            const gfwd* G = &g[ent[q] & 0x7fffffffu];
            double ex, dx, dy;
            const double alpha = alpha_of(G, (int)(ent[q] >> 31), px, py, &ex, &dx, &dy);
            for (int ch = 0; ch < 3; ++ch) acc[ch] += G->rgb[ch] * alpha * T;
            T *= 1.0 - alpha;
        }
        for (int ch = 0; ch < 3; ++ch) rgb_out[3 * i + ch] = acc[ch] + bg[ch] * T;
    }
    free(g);
    return 0;
}

/* Chain rule from the splat quantities of one Gaussian to its parameters.
 * gs = dL/d(u, v, A, B, C, alpha0, r, g, b); results are added at node n. */
static void backward_gauss(const cam64* k, const oparams64* P, int64_t n, const gfwd* g,
                           const double gs[9], double* g_mu, double* g_ls, double* g_q,
                           double* g_logit, double* g_sh)
{
    const int64_t N = P->n;
    const int K = (P->sh_degree + 1) * (P->sh_degree + 1);
    const double z = g->p[2];
    double gp[3] = {0.0, 0.0, 0.0};      /* dL / d camera-space centre */
    double gmu[3] = {0.0, 0.0, 0.0};
    /* u = fx x / z + cx, v = fy y / z + cy */
    gp[0] += gs[0] * k->fx / z;
    gp[2] -= gs[0] * k->fx * g->p[0] / (z * z);
    gp[1] += gs[1] * k->fy / z;
    gp[2] -= gs[1] * k->fy * g->p[1] / (z * z);
    /* conic (A, B, C) = (c, -b, a) / det, det = a c - b^2 */
    const double d2 = g->det * g->det;
    const double a = g->a, b = g->b, c = g->c;
    const double dA[3] = {-c * c / d2, 2.0 * b * c / d2, -b * b / d2};            /* d/d(a,b,c) */
    const double dB[3] = {b * c / d2, -(g->det + 2.0 * b * b) / d2, a * b / d2};
    const double dC[3] = {-b * b / d2, 2.0 * a * b / d2, -a * a / d2};
    double gabc[3];
    for (int i = 0; i < 3; ++i) gabc[i] = gs[2] * dA[i] + gs[3] * dB[i] + gs[4] * dC[i];
    /* Sigma_2D = M Sigma M^T (+ 0.3 I): a = S2_00, b = S2_01 = S2_10, c = S2_11 */
    const double G2[2][2] = {{gabc[0], 0.5 * gabc[1]}, {0.5 * gabc[1], gabc[2]}};
    double GS[3][3], GM[2][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int r = 0; r < 2; ++r)
                for (int s = 0; s < 2; ++s) v += g->M[r][i] * G2[r][s] * g->M[s][j];
            GS[i][j] = v;
        }
    for (int r = 0; r < 2; ++r)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int s = 0; s < 2; ++s)
                for (int a2 = 0; a2 < 3; ++a2) v += 2.0 * G2[r][s] * g->M[s][a2] * g->S[a2][j];
            GM[r][j] = v;
        }
    /* M = J W */
    double GJ[2][3];
    for (int r = 0; r < 2; ++r)
        for (int i = 0; i < 3; ++i)
            GJ[r][i] = GM[r][0] * k->W[i][0] + GM[r][1] * k->W[i][1] + GM[r][2] * k->W[i][2];
    /* J entries: fx/z, -fx tx/z^2, fy/z, -fy ty/z^2, with tx = x unless clamped
     * (then tx = +-limx z) */
    gp[2] += GJ[0][0] * (-k->fx / (z * z));
    gp[2] += GJ[1][1] * (-k->fy / (z * z));
    if (!g->clx) {
        gp[0] += GJ[0][2] * (-k->fx / (z * z));
        gp[2] += GJ[0][2] * (2.0 * k->fx * g->p[0] / (z * z * z));
    } else {
        gp[2] += GJ[0][2] * (k->fx * g->clx * k->limx / (z * z));
    }
    if (!g->cly) {
        gp[1] += GJ[1][2] * (-k->fy / (z * z));
        gp[2] += GJ[1][2] * (2.0 * k->fy * g->p[1] / (z * z * z));
    } else {
        gp[2] += GJ[1][2] * (k->fy * g->cly * k->limy / (z * z));
    }
    /* p = W mu + t */
    for (int j = 0; j < 3; ++j) gmu[j] += k->W[0][j] * gp[0] + k->W[1][j] * gp[1] + k->W[2][j] * gp[2];
    /* Sigma = R diag(s2) R^T */
    double GR[3][3];
    for (int i = 0; i < 3; ++i)
        for (int m = 0; m < 3; ++m) {
            double v = 0.0;
            for (int j = 0; j < 3; ++j) v += GS[i][j] * g->R[j][m];
            GR[i][m] = 2.0 * v * g->s2[m];
        }
    for (int m = 0; m < 3; ++m) {
        double v = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) v += g->R[i][m] * GS[i][j] * g->R[j][m];
        g_ls[m * N + n] += v * 2.0 * g->s2[m];
    }
    /* R(qh): partial derivatives of each entry */
    const double w = g->qh[0], x = g->qh[1], y = g->qh[2], zq = g->qh[3];
    double dR[4][3][3] = {
        {{0, -2 * zq, 2 * y}, {2 * zq, 0, -2 * x}, {-2 * y, 2 * x, 0}},                 /* d/dw */
        {{0, 2 * y, 2 * zq}, {2 * y, -4 * x, -2 * w}, {2 * zq, 2 * w, -4 * x}},         /* d/dx */
        {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * zq}, {-2 * w, 2 * zq, -4 * y}},         /* d/dy */
        {{-4 * zq, -2 * w, 2 * x}, {2 * w, -4 * zq, 2 * y}, {2 * x, 2 * y, 0}}};        /* d/dz */
    double gqh[4];
    for (int e = 0; e < 4; ++e) {
        double v = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) v += GR[i][j] * dR[e][i][j];
        gqh[e] = v;
    }
    /* qh = q / |q| */
    const double dot = gqh[0] * g->qh[0] + gqh[1] * g->qh[1] + gqh[2] * g->qh[2] + gqh[3] * g->qh[3];
    for (int e = 0; e < 4; ++e) g_q[e * N + n] += (gqh[e] - g->qh[e] * dot) / g->qn;
    /* alpha0 = sigmoid(l) */
    if (!g->l_clamped) g_logit[n] += gs[5] * g->a0 * (1.0 - g->a0);
    /* colour */
    double Jy[16][3];
    sh_basis_jac(P->sh_degree, g->dir, Jy);
    const double* cf = P->sh + (size_t)n * K * 3;
    double gdir[3] = {0.0, 0.0, 0.0};
    for (int ch = 0; ch < 3; ++ch) {
        const double gpre = g->pre[ch] > 0.0 ? gs[6 + ch] : 0.0;
        for (int kk = 0; kk < K; ++kk) {
            g_sh[((size_t)n * K + kk) * 3 + ch] += g->Y[kk] * gpre;
            for (int i = 0; i < 3; ++i) gdir[i] += cf[3 * kk + ch] * gpre * Jy[kk][i];
        }
    }
    /* dir = (mu - campos) / |mu - campos| */
    const double dd = gdir[0] * g->dir[0] + gdir[1] * g->dir[1] + gdir[2] * g->dir[2];
    for (int i = 0; i < 3; ++i) gmu[i] += (gdir[i] - g->dir[i] * dd) / g->dlen;
    for (int i = 0; i < 3; ++i) g_mu[i * N + n] += gmu[i];
}

int oracle_diff_grad(const ocam* c, const double bg[3], const oparams64* P, const uint32_t* sel,
                     int32_t M, const int64_t* pix, int64_t n_pix, const int64_t* offs,
                     const uint32_t* ent, const double* dL, double* g_mu, double* g_ls,
                     double* g_q, double* g_logit, double* g_sh)
{
    cam64 k;
    gfwd* g;
    if (prepare(c, P, sel, M, &k, &g)) return -1;
    double* gs = (double*)calloc((size_t)(M > 0 ? M : 1) * 9, sizeof(double));
    int64_t cap = 1;
    for (int64_t i = 0; i < n_pix; ++i)
        if (offs[i + 1] - offs[i] > cap) cap = offs[i + 1] - offs[i];
    double* Ti = (double*)malloc((size_t)cap * sizeof(double));
    double* al = (double*)malloc((size_t)cap * sizeof(double));
    double* exs = (double*)malloc((size_t)cap * sizeof(double));
    if (!gs || !Ti || !al || !exs) {
        free(g); free(gs); free(Ti); free(al); free(exs);
        return -1;
    }
    for (int64_t i = 0; i < n_pix; ++i) {
        const double px = (double)(pix[i] % c->width) + 0.5, py = (double)(pix[i] / c->width) + 0.5;
        const int64_t b = offs[i], e = offs[i + 1];
        /* forward: transmittance before each contributor */
        double T = 1.0;
        for (int64_t q = b; q < e; ++q) {
            double dx, dy;
            al[q - b] = alpha_of(&g[ent[q] & 0x7fffffffu], (int)(ent[q] >> 31), px, py, &exs[q - b],
                                 &dx, &dy);
            Ti[q - b] = T;
            T *= 1.0 - al[q - b];
        }
        /* backward: behind[ch] = sum over later contributors of c alpha T, plus bg T_final */
        double behind[3] = {bg[0] * T, bg[1] * T, bg[2] * T};
        const double* w = dL + 3 * i;
        for (int64_t q = e - 1; q >= b; --q) {
            const uint32_t m = ent[q] & 0x7fffffffu;
            const int clamped = (int)(ent[q] >> 31);
            const gfwd* G = &g[m];
            const double alpha = al[q - b], Tq = Ti[q - b];
            double galpha = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                gs[9 * m + 6 + ch] += w[ch] * alpha * Tq;
                galpha += w[ch] * (G->rgb[ch] * Tq - behind[ch] / (1.0 - alpha));
            }
            for (int ch = 0; ch < 3; ++ch) behind[ch] += G->rgb[ch] * alpha * Tq;
            if (clamped) continue;
            const double dx = G->u - px, dy = G->v - py;
            const double gpow = galpha * alpha;          /* d alpha / d power = alpha */
            gs[9 * m + 5] += galpha * exs[q - b];        /* d alpha / d alpha0 = e^power */
            gs[9 * m + 0] += gpow * (-G->A * dx - G->B * dy);
            gs[9 * m + 1] += gpow * (-G->C * dy - G->B * dx);
            gs[9 * m + 2] += gpow * (-0.5 * dx * dx);
            gs[9 * m + 3] += gpow * (-dx * dy);
            gs[9 * m + 4] += gpow * (-0.5 * dy * dy);
        }
    }
    for (int32_t m = 0; m < M; ++m)
        backward_gauss(&k, P, sel[m], &g[m], gs + 9 * m, g_mu, g_ls, g_q, g_logit, g_sh);
    free(g);
    free(gs);
    free(Ti);
    free(al);
    free(exs);
    return 0;
}
