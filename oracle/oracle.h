/*
 * CPU oracle of the FilterGS per-frame LoD render path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, deliberately unoptimised
 * restatement of what the render path computes, used to check the CUDA path.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library; the only thing both sides share is the seeded input
 * generator (the Python module that draws trees and cameras).
 *
 * Precision: every quantity that decides an integer result (frustum test,
 * R&L predicate, tile rectangle, depth key, shrink radius, the skip / stop
 * decisions of blending) is computed in IEEE binary32 with one fixed operation
 * order and no fused multiply-add (the file is compiled with
 * -ffp-contract=off).  Colours, images and KPC / GTC sums are accumulated in
 * binary64.
 *
 * Layouts (all arrays are caller-owned, row-major C order):
 *   mu[3][N], cov[6][N] (xx,xy,xz,yy,yz,zz), opacity[N], ln_opacity[N],
 *   sh[N][(deg+1)^2][3], parent[N] (-1 = root), is_leaf[N], ap[D][N]
 *   (0xFFFFFFFF past the root).
 *   splat[M][ORACLE_SPLAT_STRIDE] (see ORACLE_SPLAT_* below), rect[M][4] =
 *   x0, x1, y0, y1 (half-open tile ranges).
 *
 * Threads: built with OpenMP, the loops over nodes, selected Gaussians, tiles
 * and pixels are shared among threads; results are bit-identical to one
 * thread (no sum changes its order).  oracle_set_threads(n) sets the count
 * (n <= 0 leaves it) and returns the count in use (1 without OpenMP).
 */
#ifndef FILTERGS_ORACLE_H
#define FILTERGS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n;            /* nodes */
    int32_t depth;        /* rows of ap */
    int32_t sh_degree;    /* 0..3 */
    const float* mu;
    const float* cov;
    const float* opacity;
    const float* ln_opacity;
    const float* sh;
    const int32_t* parent;
    const uint8_t* is_leaf;
    const uint32_t* ap;
} otree;

typedef struct {
    float R[9];           /* world -> camera rotation, row-major */
    float t[3];
    float fx, fy, cx, cy;
    float tan_half_x, tan_half_y;
    float campos[3];
    int32_t width, height;
} ocam;

typedef struct {
    float tau_R;          /* R&L pixel-radius threshold (§3.2) */
    int32_t shrink;       /* 0: 3-sigma footprint, 1: shrink to opacity tau (§3.3) */
    float tau, ln_tau;    /* shrink threshold and its natural log */
    int32_t tile_w, tile_h;  /* powers of two */
    float bg[3];
} oparams;

enum {
    ORACLE_SPLAT_U = 0, ORACLE_SPLAT_V, ORACLE_SPLAT_A, ORACLE_SPLAT_B, ORACLE_SPLAT_C,
    ORACLE_SPLAT_LTHR, ORACLE_SPLAT_A0, ORACLE_SPLAT_DEPTH, ORACLE_SPLAT_R,
    ORACLE_SPLAT_G, ORACLE_SPLAT_BL, ORACLE_SPLAT_RADIUS, ORACLE_SPLAT_STRIDE
};

/* exp(x) by Cody-Waite reduction and a degree-7 Taylor polynomial (binary32). */
float oracle_expf(float x);

/* Real spherical-harmonic basis (Condon-Shortley phase) up to degree 3 at a unit
 * direction, binary64; writes (deg+1)^2 values. */
void oracle_sh_basis(int deg, const double dir[3], double* out);

/* R&L predicate P(n) of §3.2 for every node; radius_out[n] = 3*sqrt(lambda_max)
 * (NaN when out of frustum).  Returns 0. */
int oracle_set_threads(int n);

int oracle_predicate(const otree* t, const ocam* c, float tau_R, uint8_t* P_out,
                     float* radius_out);

/* Serial top-down traversal: the LoD cut as ascending node ids.  Returns M. */
int32_t oracle_filter_dfs(const otree* t, const ocam* c, float tau_R, uint32_t* sel_out);

/* Set definition {n : P(n) and no ancestor in AP(n) has P}.  Returns M. */
int32_t oracle_filter_setdef(const otree* t, const ocam* c, float tau_R, uint32_t* sel_out);

/* Projection, SH colour and footprint of the selected nodes.  rect rows of
 * Gaussians that emit no pair are {0,0,0,0}.  Returns the pair count N_P. */
int64_t oracle_project(const otree* t, const ocam* c, const oparams* p, const uint32_t* sel,
                       int32_t M, float* splat_out, int32_t* rect_out);

/* All (tile, Gaussian) pairs of the rectangles, keyed (tile << 32 | depth bits),
 * value = selected rank, sorted by (key, value).  Returns N_P, or -1 if cap is
 * too small. */
int64_t oracle_pairs(const float* splat, const int32_t* rect, int32_t M, int32_t tiles_x,
                     uint64_t* keys_out, uint32_t* vals_out, int64_t cap);

/* Pair count by testing every tile of the grid against every footprint box. */
int64_t oracle_count_pairs_bruteforce(const ocam* c, const oparams* p, const float* splat,
                                      const uint8_t* emits, int32_t M);

/* Per-pixel front-to-back blending (Eq. 2) over the sorted pairs.
 * rgb_out[3][H][W], T_out[H][W].  kpc_out (may be NULL) receives, per sorted
 * pair, the KPC of Eq. 5.  Returns 0. */
int oracle_render(const ocam* c, const oparams* p, const float* splat, const uint64_t* keys,
                  const uint32_t* vals, int64_t n_pairs, double* rgb_out, float* T_out,
                  double* kpc_out);

/* Render restricted to the listed pixels (linear indices y*W+x): rgb_out[k][3], T_out[k]. */
int oracle_render_pixels(const ocam* c, const oparams* p, const float* splat,
                         const uint64_t* keys, const uint32_t* vals, int64_t n_pairs,
                         const int64_t* pix, int64_t n_pix, double* rgb_out, float* T_out);

/* GTC per tile (Eq. 6; NaN for tiles without pairs) and the view average of
 * Eq. 7 over tiles that have pairs.  Returns the number of such tiles. */
int32_t oracle_gtc(const uint64_t* keys, const double* kpc, int64_t n_pairs, int32_t n_tiles,
                   double* G_out, double* Gbar_out);

/* The contributors of each listed pixel (linear indices y*W+x), in blending
 * order: splat rank | (alpha clamped at 0.99) << 31, for the pairs the Eq. 2
 * walk adds before it stops.  offs_out[n_pix + 1] (may be NULL) indexes
 * ent_out (may be NULL: count only).  Returns the number of entries. */
int64_t oracle_trace_pixels(const ocam* c, const oparams* p, const float* splat,
                            const uint64_t* keys, const uint32_t* vals, int64_t n_pairs,
                            const int64_t* pix, int64_t n_pix, int64_t* offs_out,
                            uint32_t* ent_out);

/* ---- differentiable form (oracle_grad.c) ---------------------------- */

/* Gaussian parameters in binary64: mu[3][n], log_scale[3][n], quat[4][n]
 * (w, x, y, z; any non-zero norm), logit[n], sh[n][(deg+1)^2][3]. */
typedef struct {
    int32_t n;
    int32_t sh_degree;
    const double* mu;
    const double* log_scale;
    const double* quat;
    const double* logit;
    const double* sh;
} oparams64;

/* ln x (binary32, positive normal x), fixed operation order. */
float oracle_lnf(float x);

/* Binary32 attributes from binary32 parameters (n nodes): cov[6][n],
 * opacity[n] = sigmoid(l), ln_opacity[n] = -ln(1 + e^{-l}), l clamped to
 * [-80, 80]. */
void oracle_prep_params(int32_t n, const float* log_scale, const float* quat, const float* logit,
                        float* cov_out, float* opacity_out, float* ln_opacity_out);

/* Image of the listed pixels as a binary64 function of the parameters, with
 * the cut sel[M] and the contributor lists (oracle_trace_pixels) frozen:
 * rgb_out[n_pix][3].  Returns 0, -1 if out of memory. */
int oracle_diff_render(const ocam* c, const double bg[3], const oparams64* P, const uint32_t* sel,
                       int32_t M, const int64_t* pix, int64_t n_pix, const int64_t* offs,
                       const uint32_t* ent, double* rgb_out);

/* Gradient of L = sum_i dL[i][ch] rgb[i][ch] for that function, ADDED to
 * g_mu[3][n], g_ls[3][n], g_q[4][n], g_logit[n], g_sh[n][K][3].  Returns 0,
 * -1 if out of memory. */
int oracle_diff_grad(const ocam* c, const double bg[3], const oparams64* P, const uint32_t* sel,
                     int32_t M, const int64_t* pix, int64_t n_pix, const int64_t* offs,
                     const uint32_t* ent, const double* dL, double* g_mu, double* g_ls,
                     double* g_q, double* g_logit, double* g_sh);

#ifdef __cplusplus
}
#endif
#endif
