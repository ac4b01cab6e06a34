/*
 * CPU oracle of the FilterGS per-frame LoD render path.
 *
 * TEST INFRASTRUCTURE ONLY: see oracle.h.  Plain serial C, written to be read
 * against the paper: §3.2 (R&L filter, Ancestor filter, LoD cut), Eq. 1-2
 * (Gaussian and front-to-back blending), §3.3 (KPC Eq. 5, GTC Eq. 6-7,
 * shrink radius and tau Eq. 8).  Readings of passages the paper leaves open
 * are noted where they are used.
 *
 * Must be compiled with -ffp-contract=off and without -ffast-math.
 *
 * Optional OpenMP (when built with -fopenmp): loops over nodes, selected
 * Gaussians, tiles and pixels run in parallel.  Every parallel iteration
 * writes its own outputs and each sum keeps its serial order (KPC is summed
 * per tile, over the tile's pixels in row-major order, exactly as the serial
 * loop over the image adds them), so results are bit-identical to one thread.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define ALPHA_MAX 0.99f                     /* opacity clamp */
#define ALPHA_MIN_LN 5.5412635451584258f   /* ln 255: skip below alpha 1/255 */
#define T_STOP 0.0001f                      /* stop once T would fall below 1e-4 */
#define Z_NEAR 0.2f
#define FRUSTUM_GUARD 1.3f
#define LOWPASS 0.3f

/* ------------------------------------------------------------------ */
/* exp                                                                */
/* ------------------------------------------------------------------ */

/* e^x for binary32.  Argument reduction after Cody & Waite (Software Manual
 * for the Elementary Functions, 1980): k = the integer nearest to x / ln 2,
 * taken from the binary32 sum x log2(e) + 1.5 * 2^23 formed with one rounding
 * (a fused multiply-add), and r = x - k ln 2 with ln 2 split into a short
 * leading part (exact products for |k| < 2^15) plus a correction.  e^r,
 * |r| <= ln2/2, is the Taylor polynomial of degree 7 by Horner's rule with
 * fused multiply-adds (truncation < 6e-9 relative), scaled by 2^k built from
 * its exponent bits.  Every step is an IEEE 754 binary32 operation (fmaf is
 * IEEE fusedMultiplyAdd) in a fixed order, so any conforming machine returns
 * the same bits. */
float oracle_expf(float x)
{
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return INFINITY;
    const float t = fmaf(x, 1.44269504088896341f, 12582912.0f);
    const float kf = t - 12582912.0f;
    float r = fmaf(kf, -0.693359375f, x);
    r = fmaf(kf, 2.12194440e-4f, r);
    float p = 1.98412698412698413e-4f;            /* 1/7! */
    p = fmaf(p, r, 1.38888888888888889e-3f);      /* 1/6! */
    p = fmaf(p, r, 8.33333333333333333e-3f);      /* 1/5! */
    p = fmaf(p, r, 4.16666666666666667e-2f);      /* 1/4! */
    p = fmaf(p, r, 1.66666666666666667e-1f);      /* 1/3! */
    p = fmaf(p, r, 0.5f);                         /* 1/2! */
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    const int32_t k = (int32_t)kf;
    const uint32_t bits = (uint32_t)(k + 127) << 23;
    float two_k;
    memcpy(&two_k, &bits, sizeof two_k);
    return p * two_k;
}

/* ------------------------------------------------------------------ */
/* spherical harmonics                                                */
/* ------------------------------------------------------------------ */

/* Real spherical harmonics Y_lm (Condon-Shortley phase), written in Cartesian
 * form for a unit direction (x, y, z), ordered m = -l..l within each degree.
 * Normalisation constants are the textbook closed forms. */
void oracle_sh_basis(int deg, const double dir[3], double* out)
{
    const double pi = 3.14159265358979323846;
    const double x = dir[0], y = dir[1], z = dir[2];
    out[0] = 0.5 * sqrt(1.0 / pi);
    if (deg < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    out[1] = -k1 * y;
    out[2] = k1 * z;
    out[3] = -k1 * x;
    if (deg < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    out[4] = k2a * x * y;
    out[5] = -k2a * y * z;
    out[6] = k2b * (2.0 * z * z - x * x - y * y);
    out[7] = -k2a * x * z;
    out[8] = k2c * (x * x - y * y);
    if (deg < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    out[9] = -k3a * y * (3.0 * x * x - y * y);
    out[10] = k3b * x * y * z;
    out[11] = -k3c * y * (4.0 * z * z - x * x - y * y);
    out[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    out[13] = -k3c * x * (4.0 * z * z - x * x - y * y);
    out[14] = k3e * z * (x * x - y * y);
    out[15] = -k3a * x * (x * x - 3.0 * y * y);
}

/* ------------------------------------------------------------------ */
/* screen-space covariance (EWA splatting)                            */
/* ------------------------------------------------------------------ */

typedef struct {
    int in_frustum;
    float vx, vy, vz;      /* camera-space centre */
    float a, b, c;         /* Sigma_2D = [[a b][b c]] incl. the 0.3 low-pass */
    float lam;             /* larger eigenvalue of Sigma_2D */
} oview;

/* Camera-space centre, frustum test and Sigma_2D = J W Sigma W^T J^T + 0.3 I of
 * one node.  "In-frustum" (§3.2) is read as: depth above 0.2 and the centre
 * within 1.3x the half-FOV tangents; J uses the same clamped tangents. */
static oview view_node(const otree* t, const ocam* cam, int64_t n)
{
    oview o;
    const int64_t N = t->n;
    const float mx = t->mu[n], my = t->mu[N + n], mz = t->mu[2 * N + n];
    const float* R = cam->R;
    o.vx = ((R[0] * mx + R[1] * my) + R[2] * mz) + cam->t[0];
    o.vy = ((R[3] * mx + R[4] * my) + R[5] * mz) + cam->t[1];
    o.vz = ((R[6] * mx + R[7] * my) + R[8] * mz) + cam->t[2];
    const float limx = FRUSTUM_GUARD * cam->tan_half_x;
    const float limy = FRUSTUM_GUARD * cam->tan_half_y;
    o.in_frustum = 0;
    o.a = o.b = o.c = o.lam = 0.0f;
    if (!(o.vz > Z_NEAR)) return o;
    const float txtz = o.vx / o.vz;
    const float tytz = o.vy / o.vz;
    if (!(txtz >= -limx && txtz <= limx && tytz >= -limy && tytz <= limy)) return o;
    o.in_frustum = 1;

    float clx = txtz < -limx ? -limx : txtz;
    clx = clx > limx ? limx : clx;
    float cly = tytz < -limy ? -limy : tytz;
    cly = cly > limy ? limy : cly;
    const float txc = clx * o.vz;
    const float tyc = cly * o.vz;
    const float tz2 = o.vz * o.vz;
    const float j00 = cam->fx / o.vz;
    const float j11 = cam->fy / o.vz;
    const float j02 = -((cam->fx * txc) / tz2);
    const float j12 = -((cam->fy * tyc) / tz2);
    /* M = J W: rows m0, m1 (2x3) */
    const float m00 = j00 * R[0] + j02 * R[6];
    const float m01 = j00 * R[1] + j02 * R[7];
    const float m02 = j00 * R[2] + j02 * R[8];
    const float m10 = j11 * R[3] + j12 * R[6];
    const float m11 = j11 * R[4] + j12 * R[7];
    const float m12 = j11 * R[5] + j12 * R[8];
    const float s00 = t->cov[n], s01 = t->cov[N + n], s02 = t->cov[2 * N + n];
    const float s11 = t->cov[3 * N + n], s12 = t->cov[4 * N + n], s22 = t->cov[5 * N + n];
    const float u0 = (s00 * m00 + s01 * m01) + s02 * m02;
    const float u1 = (s01 * m00 + s11 * m01) + s12 * m02;
    const float u2 = (s02 * m00 + s12 * m01) + s22 * m02;
    const float w0 = (s00 * m10 + s01 * m11) + s02 * m12;
    const float w1 = (s01 * m10 + s11 * m11) + s12 * m12;
    const float w2 = (s02 * m10 + s12 * m11) + s22 * m12;
    o.a = ((m00 * u0 + m01 * u1) + m02 * u2) + LOWPASS;
    o.b = (m10 * u0 + m11 * u1) + m12 * u2;
    o.c = ((m10 * w0 + m11 * w1) + m12 * w2) + LOWPASS;
    const float det = o.a * o.c - o.b * o.b;
    const float mid = 0.5f * (o.a + o.c);
    float disc = mid * mid - det;
    disc = disc > 0.1f ? disc : 0.1f;
    o.lam = mid + sqrtf(disc);
    return o;
}

/* ------------------------------------------------------------------ */
/* §3.2 filters                                                       */
/* ------------------------------------------------------------------ */

/* R&L filter: keep an in-frustum node if it is a leaf, or if its pixel radius
 * R_2D = 3 sigma, sigma = sqrt(lambda_max) (the larger screen-space standard
 * deviation), is at most tau_R.  Out-of-frustum nodes fail. */
int oracle_predicate(const otree* t, const ocam* c, float tau_R, uint8_t* P_out,
                     float* radius_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < t->n; ++n) {
        oview o = view_node(t, c, n);
        float R2d = o.in_frustum ? 3.0f * sqrtf(o.lam) : NAN;
        if (radius_out) radius_out[n] = R2d;
        P_out[n] = (uint8_t)(o.in_frustum && (t->is_leaf[n] || R2d <= tau_R));
    }
    return 0;
}

static int cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

typedef struct {
    const int64_t* first;   /* CSR offsets of children, n+1 */
    const uint32_t* kids;
    const uint8_t* P;
    uint32_t* out;
    int32_t m;
} dfs_state;

static void dfs_visit(dfs_state* s, uint32_t n)
{
    if (s->P[n]) {
        s->out[s->m++] = n;
        return;
    }
    for (int64_t k = s->first[n]; k < s->first[n + 1]; ++k) dfs_visit(s, s->kids[k]);
}

/* Serial LoD traversal: from the root, keep a node that passes R&L and stop,
 * otherwise descend into its children (in id order).  A culled internal node
 * does not prune its subtree.  Output sorted ascending. */
int32_t oracle_filter_dfs(const otree* t, const ocam* c, float tau_R, uint32_t* sel_out)
{
    const int64_t N = t->n;
    uint8_t* P = (uint8_t*)malloc((size_t)N);
    int64_t* first = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    uint32_t* kids = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(N > 0 ? N : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
    oracle_predicate(t, c, tau_R, P, NULL);
    for (int64_t n = 0; n < N; ++n)
        if (t->parent[n] >= 0) first[t->parent[n] + 1]++;
    for (int64_t n = 0; n < N; ++n) first[n + 1] += first[n];
    memcpy(fill, first, sizeof(int64_t) * (size_t)(N + 1));
    for (int64_t n = 0; n < N; ++n)
        if (t->parent[n] >= 0) kids[fill[t->parent[n]]++] = (uint32_t)n;
    dfs_state s = {first, kids, P, sel_out, 0};
    for (int64_t n = 0; n < N; ++n)
        if (t->parent[n] < 0) dfs_visit(&s, (uint32_t)n);
    qsort(sel_out, (size_t)s.m, sizeof(uint32_t), cmp_u32);
    free(P); free(first); free(kids); free(fill);
    return s.m;
}

/* Ancestor filter over the precomputed ancestor paths: a node that passes R&L
 * is dropped if any node of AP(n) (parent up to the root) also passes. */
int32_t oracle_filter_setdef(const otree* t, const ocam* c, float tau_R, uint32_t* sel_out)
{
    const int64_t N = t->n;
    uint8_t* P = (uint8_t*)malloc((size_t)N);
    oracle_predicate(t, c, tau_R, P, NULL);
    int32_t m = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (!P[n]) continue;
        int blocked = 0;
        for (int32_t k = 0; k < t->depth; ++k) {
            uint32_t a = t->ap[(int64_t)k * N + n];
            if (a == 0xFFFFFFFFu) break;
            if (P[a]) { blocked = 1; break; }
        }
        if (!blocked) sel_out[m++] = (uint32_t)n;
    }
    free(P);
    return m;
}

/* ------------------------------------------------------------------ */
/* projection, colour, footprint (§3.3 shrinking)                      */
/* ------------------------------------------------------------------ */

static float clampf(float v, float lo, float hi)
{
    v = v < lo ? lo : v;
    return v > hi ? hi : v;
}

int64_t oracle_project(const otree* t, const ocam* c, const oparams* p, const uint32_t* sel,
                       int32_t M, float* splat_out, int32_t* rect_out)
{
    const int64_t N = t->n;
    const int K = (t->sh_degree + 1) * (t->sh_degree + 1);
    const int32_t tiles_x = (c->width + p->tile_w - 1) / p->tile_w;
    const int32_t tiles_y = (c->height + p->tile_h - 1) / p->tile_h;
    int64_t n_pairs = 0;
#pragma omp parallel for schedule(static) reduction(+ : n_pairs)
    for (int32_t m = 0; m < M; ++m) {
        const int64_t n = sel[m];
        float* s = splat_out + (int64_t)m * ORACLE_SPLAT_STRIDE;
        int32_t* rc = rect_out + (int64_t)m * 4;
        oview o = view_node(t, c, n);
        for (int k = 0; k < ORACLE_SPLAT_STRIDE; ++k) s[k] = 0.0f;
        rc[0] = rc[1] = rc[2] = rc[3] = 0;
        const float u = c->fx * (o.vx / o.vz) + c->cx;
        const float v = c->fy * (o.vy / o.vz) + c->cy;
        const float det = o.a * o.c - o.b * o.b;
        s[ORACLE_SPLAT_U] = u;
        s[ORACLE_SPLAT_V] = v;
        s[ORACLE_SPLAT_DEPTH] = o.vz;
        s[ORACLE_SPLAT_A0] = t->opacity[n];
        /* skip test alpha0 * e^power < 1/255 taken in the log domain */
        s[ORACLE_SPLAT_LTHR] = -ALPHA_MIN_LN - t->ln_opacity[n];

        /* view-dependent colour: sum_lm c_lm Y_lm(d) + 0.5, clamped at 0 */
        double d[3] = {(double)t->mu[n] - c->campos[0], (double)t->mu[N + n] - c->campos[1],
                       (double)t->mu[2 * N + n] - c->campos[2]};
        const double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= dl; d[1] /= dl; d[2] /= dl;
        double Y[16];
        oracle_sh_basis(t->sh_degree, d, Y);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += Y[k] * (double)t->sh[(n * K + k) * 3 + ch];
            acc += 0.5;
            s[ORACLE_SPLAT_R + ch] = (float)(acc > 0.0 ? acc : 0.0);
        }
        if (!o.in_frustum || !(det > 0.0f)) continue;
        s[ORACLE_SPLAT_A] = o.c / det;
        s[ORACLE_SPLAT_B] = -o.b / det;
        s[ORACLE_SPLAT_C] = o.a / det;

        /* Footprint radius.  3-sigma: r = 3 sqrt(lambda_max).  Shrinking (§3.3)
         * reads sigma_max of r = sqrt(2 sigma_max ln(alpha0 / tau)) as the
         * variance lambda_max, i.e. the radius where alpha0 e^{-r^2 / 2 lambda}
         * = tau, capped at the 3-sigma radius; alpha0 <= tau emits nothing. */
        const float r3 = 3.0f * sqrtf(o.lam);
        float r = r3;
        if (p->shrink) {
            const float g = 2.0f * (t->ln_opacity[n] - p->ln_tau);
            if (!(g > 0.0f)) continue;
            if (g < 9.0f) r = sqrtf(o.lam * g);
        }
        s[ORACLE_SPLAT_RADIUS] = r;
        /* Tiles whose pixel square [tw*i, tw*(i+1)) meets [u - r, u + r]. */
        const float fx0 = clampf(floorf((u - r) / (float)p->tile_w), 0.0f, (float)tiles_x);
        const float fx1 = clampf(floorf((u + r) / (float)p->tile_w) + 1.0f, 0.0f, (float)tiles_x);
        const float fy0 = clampf(floorf((v - r) / (float)p->tile_h), 0.0f, (float)tiles_y);
        const float fy1 = clampf(floorf((v + r) / (float)p->tile_h) + 1.0f, 0.0f, (float)tiles_y);
        const int32_t x0 = (int32_t)fx0, x1 = (int32_t)fx1, y0 = (int32_t)fy0, y1 = (int32_t)fy1;
        if (x1 <= x0 || y1 <= y0) continue;
        rc[0] = x0; rc[1] = x1; rc[2] = y0; rc[3] = y1;
        n_pairs += (int64_t)(x1 - x0) * (int64_t)(y1 - y0);
    }
    return n_pairs;
}

typedef struct { uint64_t key; uint32_t val; } opair;

static int cmp_pair(const void* a, const void* b)
{
    const opair* x = (const opair*)a;
    const opair* y = (const opair*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->val > y->val) - (x->val < y->val);
}

/* One key per (Gaussian, tile) of its rectangle: (tile id << 32) | depth bits;
 * depth is positive so its bit pattern orders like the value.  Sorted by key,
 * ties by the selected rank (= ascending node id). */
int64_t oracle_pairs(const float* splat, const int32_t* rect, int32_t M, int32_t tiles_x,
                     uint64_t* keys_out, uint32_t* vals_out, int64_t cap)
{
    int64_t total = 0;
    for (int32_t m = 0; m < M; ++m) {
        const int32_t* rc = rect + (int64_t)m * 4;
        total += (int64_t)(rc[1] - rc[0]) * (int64_t)(rc[3] - rc[2]);
    }
    if (total > cap) return -1;
    opair* pr = (opair*)malloc(sizeof(opair) * (size_t)(total > 0 ? total : 1));
    /* Gaussian m's pairs start after those of Gaussians 0 .. m-1 */
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    int64_t k = 0;
    for (int32_t m = 0; m < M; ++m) {
        const int32_t* rc = rect + (int64_t)m * 4;
        start[m] = k;
        k += (int64_t)(rc[1] - rc[0]) * (int64_t)(rc[3] - rc[2]);
    }
#pragma omp parallel for schedule(static)
    for (int32_t m = 0; m < M; ++m) {
        const int32_t* rc = rect + (int64_t)m * 4;
        float depth = splat[(int64_t)m * ORACLE_SPLAT_STRIDE + ORACLE_SPLAT_DEPTH];
        uint32_t dbits;
        memcpy(&dbits, &depth, sizeof dbits);
        int64_t q = start[m];
        for (int32_t ty = rc[2]; ty < rc[3]; ++ty)
            for (int32_t tx = rc[0]; tx < rc[1]; ++tx) {
                uint64_t tile = (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                pr[q].key = (tile << 32) | dbits;
                pr[q].val = (uint32_t)m;
                ++q;
            }
    }
    free(start);
    qsort(pr, (size_t)total, sizeof(opair), cmp_pair);
    for (int64_t i = 0; i < total; ++i) {
        keys_out[i] = pr[i].key;
        vals_out[i] = pr[i].val;
    }
    free(pr);
    return total;
}

int64_t oracle_count_pairs_bruteforce(const ocam* c, const oparams* p, const float* splat,
                                      const uint8_t* emits, int32_t M)
{
    const int32_t tiles_x = (c->width + p->tile_w - 1) / p->tile_w;
    const int32_t tiles_y = (c->height + p->tile_h - 1) / p->tile_h;
    int64_t count = 0;
    for (int32_t m = 0; m < M; ++m) {
        if (!emits[m]) continue;
        const float* s = splat + (int64_t)m * ORACLE_SPLAT_STRIDE;
        const float u = s[ORACLE_SPLAT_U], v = s[ORACLE_SPLAT_V], r = s[ORACLE_SPLAT_RADIUS];
        const float xl = u - r, xh = u + r, yl = v - r, yh = v + r;
        for (int32_t ty = 0; ty < tiles_y; ++ty)
            for (int32_t tx = 0; tx < tiles_x; ++tx) {
                const float px0 = (float)(p->tile_w * tx), px1 = (float)(p->tile_w * (tx + 1));
                const float py0 = (float)(p->tile_h * ty), py1 = (float)(p->tile_h * (ty + 1));
                if (px0 <= xh && xl < px1 && py0 <= yh && yl < py1) ++count;
            }
    }
    return count;
}

/* ------------------------------------------------------------------ */
/* Eq. 2 blending and Eq. 5 KPC                                        */
/* ------------------------------------------------------------------ */

/* power = -1/2 (A dx^2 + 2 B dx dy + C dy^2) for the conic (A, B, C) of splat
 * record s, evaluated as (A' dx + B' dy) dx + (C' dy) dy with the per-Gaussian
 * coefficients A' = -A/2, B' = -B, C' = -C/2: one product for B' dy, two for
 * (C' dy) dy, then two fused multiply-adds, in that order. */
static float oracle_power(const float* s, float dx, float dy)
{
    const float Ah = -0.5f * s[ORACLE_SPLAT_A];
    const float Bn = -s[ORACLE_SPLAT_B];
    const float Ch = -0.5f * s[ORACLE_SPLAT_C];
    return fmaf(fmaf(Ah, dx, Bn * dy), dx, (Ch * dy) * dy);
}

/* Blend one pixel front to back over the pairs [b, e) of its tile.
 * 3DGS conventions: power = -1/2 d^T conic d; skip power > 0; skip alpha below
 * 1/255 (tested as power < -ln 255 - ln alpha0); alpha = min(0.99, alpha0 e^power);
 * stop, before adding, at the first Gaussian that would take T below 1e-4. */
static void blend_pixel(const float* splat, const uint32_t* vals, int64_t b, int64_t e, float px,
                        float py, double rgb[3], float* T_final, double* kpc, uint32_t* rec,
                        int64_t* n_rec)
{
    float T = 1.0f;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t q = b; q < e; ++q) {
        const float* s = splat + (int64_t)vals[q] * ORACLE_SPLAT_STRIDE;
        const float dx = s[ORACLE_SPLAT_U] - px;
        const float dy = s[ORACLE_SPLAT_V] - py;
        const float power = oracle_power(s, dx, dy);
        if (power > 0.0f) continue;
        if (power < s[ORACLE_SPLAT_LTHR]) continue;
        float alpha = s[ORACLE_SPLAT_A0] * oracle_expf(power);
        const int clamped = !(alpha < ALPHA_MAX);
        alpha = alpha < ALPHA_MAX ? alpha : ALPHA_MAX;
        const float Tn = T * (1.0f - alpha);
        if (Tn < T_STOP) break;
        if (n_rec) {
            if (rec) rec[*n_rec] = vals[q] | ((uint32_t)clamped << 31);
            ++*n_rec;
        }
        const double w = (double)alpha * (double)T;
        acc[0] += (double)s[ORACLE_SPLAT_R] * w;
        acc[1] += (double)s[ORACLE_SPLAT_G] * w;
        acc[2] += (double)s[ORACLE_SPLAT_BL] * w;
        if (kpc) kpc[q] += w;
        T = Tn;
    }
    rgb[0] = acc[0];
    rgb[1] = acc[1];
    rgb[2] = acc[2];
    *T_final = T;
}

static void tile_range(const uint64_t* keys, int64_t n_pairs, uint64_t tile, int64_t* b, int64_t* e)
{
    /* first key >= tile << 32 and first key >= (tile + 1) << 32 (binary search) */
    int64_t lo = 0, hi = n_pairs;
    const uint64_t k0 = tile << 32, k1 = (tile + 1) << 32;
    while (lo < hi) { int64_t mid = (lo + hi) / 2; if (keys[mid] < k0) lo = mid + 1; else hi = mid; }
    *b = lo;
    hi = n_pairs;
    while (lo < hi) { int64_t mid = (lo + hi) / 2; if (keys[mid] < k1) lo = mid + 1; else hi = mid; }
    *e = lo;
}

/* Every pixel blends the pairs of its own tile, so the image is rendered tile
 * by tile; within a tile, pixels go row by row (the order in which a pair's
 * KPC terms are added). */
int oracle_render(const ocam* c, const oparams* p, const float* splat, const uint64_t* keys,
                  const uint32_t* vals, int64_t n_pairs, double* rgb_out, float* T_out,
                  double* kpc_out)
{
    const int64_t W = c->width, H = c->height;
    const int32_t tiles_x = (c->width + p->tile_w - 1) / p->tile_w;
    const int32_t tiles_y = (c->height + p->tile_h - 1) / p->tile_h;
    if (kpc_out) memset(kpc_out, 0, sizeof(double) * (size_t)n_pairs);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t tile = 0; tile < (int64_t)tiles_x * tiles_y; ++tile) {
        const int64_t ty = tile / tiles_x, tx = tile % tiles_x;
        int64_t b, e;
        tile_range(keys, n_pairs, (uint64_t)tile, &b, &e);
        const int64_t y_end = (ty + 1) * p->tile_h < H ? (ty + 1) * p->tile_h : H;
        const int64_t x_end = (tx + 1) * p->tile_w < W ? (tx + 1) * p->tile_w : W;
        for (int64_t y = ty * p->tile_h; y < y_end; ++y)
            for (int64_t x = tx * p->tile_w; x < x_end; ++x) {
                double rgb[3];
                float T;
                blend_pixel(splat, vals, b, e, (float)x + 0.5f, (float)y + 0.5f, rgb, &T, kpc_out, NULL,
                            NULL);
                for (int ch = 0; ch < 3; ++ch)
                    rgb_out[ch * W * H + y * W + x] = rgb[ch] + (double)T * (double)p->bg[ch];
                T_out[y * W + x] = T;
            }
    }
    return 0;
}

int oracle_render_pixels(const ocam* c, const oparams* p, const float* splat,
                         const uint64_t* keys, const uint32_t* vals, int64_t n_pairs,
                         const int64_t* pix, int64_t n_pix, double* rgb_out, float* T_out)
{
    const int64_t W = c->width;
    const int32_t tiles_x = (c->width + p->tile_w - 1) / p->tile_w;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_pix; ++i) {
        const int64_t x = pix[i] % W, y = pix[i] / W;
        const uint64_t tile = (uint64_t)(y / p->tile_h) * (uint64_t)tiles_x + (uint64_t)(x / p->tile_w);
        int64_t b, e;
        tile_range(keys, n_pairs, tile, &b, &e);
        double rgb[3];
        float T;
        blend_pixel(splat, vals, b, e, (float)x + 0.5f, (float)y + 0.5f, rgb, &T, NULL, NULL, NULL);
        for (int ch = 0; ch < 3; ++ch) rgb_out[i * 3 + ch] = rgb[ch] + (double)T * (double)p->bg[ch];
        T_out[i] = T;
    }
    return 0;
}

int64_t oracle_trace_pixels(const ocam* c, const oparams* p, const float* splat,
                            const uint64_t* keys, const uint32_t* vals, int64_t n_pairs,
                            const int64_t* pix, int64_t n_pix, int64_t* offs_out,
                            uint32_t* ent_out)
{
    const int64_t W = c->width;
    const int32_t tiles_x = (c->width + p->tile_w - 1) / p->tile_w;
    int64_t total = 0;
    for (int64_t i = 0; i < n_pix; ++i) {
        const int64_t x = pix[i] % W, y = pix[i] / W;
        const uint64_t tile = (uint64_t)(y / p->tile_h) * (uint64_t)tiles_x + (uint64_t)(x / p->tile_w);
        int64_t b, e;
        tile_range(keys, n_pairs, tile, &b, &e);
        double rgb[3];
        float T;
        if (offs_out) offs_out[i] = total;
        /* appends this pixel's contributors at ent_out[total ...] and advances total */
        blend_pixel(splat, vals, b, e, (float)x + 0.5f, (float)y + 0.5f, rgb, &T, NULL, ent_out,
                    &total);
    }
    if (offs_out) offs_out[n_pix] = total;
    return total;
}

/* Eq. 6: G_i = mean KPC over the n_gs pairs keyed to tile i.  Eq. 7: the view
 * average over tiles; a tile with no pair has no G (0/0) and is left out. */
int32_t oracle_gtc(const uint64_t* keys, const double* kpc, int64_t n_pairs, int32_t n_tiles,
                   double* G_out, double* Gbar_out)
{
    double* sum = (double*)calloc((size_t)n_tiles, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)n_tiles, sizeof(int64_t));
    for (int64_t q = 0; q < n_pairs; ++q) {
        const int64_t tile = (int64_t)(keys[q] >> 32);
        sum[tile] += kpc[q];
        cnt[tile] += 1;
    }
    double total = 0.0;
    int32_t used = 0;
    for (int32_t i = 0; i < n_tiles; ++i) {
        if (cnt[i] > 0) {
            G_out[i] = sum[i] / (double)cnt[i];
            total += G_out[i];
            ++used;
        } else {
            G_out[i] = NAN;
        }
    }
    *Gbar_out = used > 0 ? total / (double)used : NAN;
    free(sum);
    free(cnt);
    return used;
}
