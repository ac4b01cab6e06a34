/*
 * filtergs.h -- C ABI of the GB300 (sm_103a) FilterGS LoD render path.
 *
 * The library renders a Level-of-Detail 3D Gaussian Splatting tree for one
 * camera per call, following FilterGS (traversal-free parallel filtering and
 * scene-adaptive Gaussian shrinking):
 *   (a) R&L filter + Ancestor filter over precomputed ancestor paths (§3.2),
 *   (b) compaction of the survivors, EWA projection and SH colour (§3.1),
 *   (c) footprint shrinking to opacity tau (§3.3, Eq. 8), Gaussian-tile pairs
 *       ordered by (tile, depth, rank): per-tile pair counts, tile ranges, a
 *       scatter of the pairs into per-tile buckets and a sort of each bucket,
 *   (d) per-tile front-to-back alpha blending (Eq. 2),
 * plus the scene calibration that derives tau from the GTC metric (Eq. 5-8).
 * Every step runs in hand-written CUDA kernels; there is no CPU fallback.
 *
 * Conventions
 *  - Every call returns an int status: FGS_OK (0) or a negative FGS_ERR_*.
 *    fgs_last_error() gives a context-owned message for the last failure.
 *    No C++ exception crosses this boundary.
 *  - A context is bound to one CUDA device.  It owns all device memory it
 *    allocates (tree copy, frame buffers) and frees it in fgs_destroy().
 *    Frame calls allocate nothing once capacities are reserved: buffers are
 *    (re)allocated only in fgs_create(), fgs_load_tree(), fgs_set_camera()
 *    (larger image) and fgs_set_params() (new pair capacity).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream); every kernel and copy of a call is enqueued on it.  Calls whose
 *    outputs are device pointers are asynchronous; calls writing host
 *    pointers synchronise the stream before returning.
 *  - Errors raised on the device (pair capacity exceeded, a bounded spin-wait
 *    that timed out) are latched in a device status word and returned by the
 *    next synchronising call or fgs_sync().  After FGS_ERR_TIMEOUT from a
 *    render (a blend's staging copy whose wait gave up may still have been in
 *    flight when its block exited) the frame and the context are not to be
 *    trusted: destroy the context.  (fgs_probe_wait_timeout's timeout is the
 *    exception: its wait has no copy in flight.)
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef FILTERGS_H
#define FILTERGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGS_VERSION 3

#define FGS_OK 0
#define FGS_ERR_ARG (-1)       /* invalid argument (NULL, size, NaN camera ...) */
#define FGS_ERR_TREE (-2)      /* tree failed validation */
#define FGS_ERR_CUDA (-3)      /* CUDA runtime error */
#define FGS_ERR_CAPACITY (-4)  /* pair or selection capacity exceeded on the device */
#define FGS_ERR_TIMEOUT (-5)   /* a bounded device spin-wait gave up */
#define FGS_ERR_STATE (-6)     /* call out of order (no tree, no camera ...) */
#define FGS_ERR_NOMEM (-7)     /* device allocation failed */

#define FGS_SHRINK_OFF 0       /* 3-sigma footprint */
#define FGS_SHRINK_ON 1        /* footprint where opacity decays to tau (§3.3) */

/* fgs_render flags */
#define FGS_RENDER_STATS 1u        /* fill M and N_P in fgs_stats (synchronises) */
#define FGS_RENDER_STAGE_EVENTS 2u /* record per-stage CUDA events (see fgs_stage_times) */
#define FGS_RENDER_COUNT 8u        /* count the blend's work (fgs_stats blend_*); implies STATS */
#define FGS_RENDER_KEEP 16u        /* keep per-pixel final T and stop position (8 bytes a pixel,
                                      context-owned) so that fgs_backward need not recompute
                                      them; ignored with COUNT */
#define FGS_RENDER_ASYNC 32u       /* host outputs without waiting: the image is copied to the
                                      host buffers on a context-owned copy stream while the
                                      caller's stream goes on with the next frame (two frames in
                                      flight, two context-owned device images); the buffers hold
                                      the frame once fgs_sync returns; not with STATS / COUNT */

#define FGS_N_STAGES 7             /* filter R&L, ancestor filter + compaction, projection + per-tile
                                      pair counts, tile ranges, key scatter, per-tile sort, blend */

/* fgs_render_batch flags (FGS_RENDER_STATS also applies) */
#define FGS_BATCH_GRAPH 4u         /* replay the batch as one captured CUDA graph */

typedef struct fgs_ctx fgs_ctx;

/* LoD tree in structure-of-arrays form, HOST pointers (§3.1 "Hierarchical
 * Gaussian Tree"; ancestor paths AP of §3.2).  N = n_nodes, D = depth,
 * K = (sh_degree + 1)^2.
 *   mu[3][N]          centres
 *   cov[6][N]         covariance upper triangle xx, xy, xz, yy, yz, zz
 *   opacity[N]        alpha_0 in (0, 1]
 *   ln_opacity[N]     ln alpha_0 (the shrink test compares logs, so no
 *                     transcendental decides a footprint)
 *   sh[N][K][3]       SH coefficients, real basis with Condon-Shortley phase
 *   parent[N]         parent id, -1 for the (single) root
 *   is_leaf[N]        1 for a leaf (no children), else 0
 *   ap[D][N]          row k = (k+1)-th ancestor of each node, 0xFFFFFFFF past
 *                     the root; must equal the parent chain.
 * The arrays are read during fgs_load_tree() only (copied to the device). */
typedef struct fgs_tree {
    uint32_t n_nodes;
    uint32_t depth;
    uint32_t sh_degree;
    uint32_t reserved;
    const float* mu;
    const float* cov;
    const float* opacity;
    const float* ln_opacity;
    const float* sh;
    const int32_t* parent;
    const uint8_t* is_leaf;
    const uint32_t* ap;
} fgs_tree;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  v = R x + t maps
 * world to camera (R row-major).  Pixel (i, j) samples at (i + 0.5, j + 0.5);
 * a centre projects to (fx vx/vz + cx, fy vy/vz + cy).  tan_half_x/y are the
 * half-FOV tangents (the frustum test allows 1.3x of them). */
typedef struct fgs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float tan_half_x, tan_half_y;
    float campos[3];
    int32_t width, height;
} fgs_camera;

typedef struct fgs_params {
    float tau_R;              /* R&L pixel-radius threshold, 3 px in the paper (§3.2) */
    int32_t tile_w, tile_h;   /* tile size in pixels: 64x4, 32x8, 16x16 (default) or 8x32 */
    float bg[3];              /* background colour added as T * bg */
    uint64_t pair_capacity;   /* max Gaussian-tile pairs per frame (0 = keep current / default) */
    int32_t blend_warp_w;     /* blend block shape: warps of 8x4 (8, default; 0 = 8) or 4x8 (4) pixels */
    int32_t reserved;
} fgs_params;

typedef struct fgs_stats {
    uint32_t n_selected;      /* M: nodes in the LoD cut */
    uint32_t n_emitting;      /* selected Gaussians with at least one pair (fgs_render) */
    uint64_t n_pairs;         /* N_P: Gaussian-tile pairs (may exceed capacity on error) */
    uint32_t n_launches;      /* kernels this call enqueued */
    int32_t device_status;    /* latched device status (FGS_OK if none) */
    uint64_t blend_entries;   /* FGS_RENDER_COUNT: lockstep warp steps of the blend's list walk
                                 (a step tests one list entry in each half of a warp) */
    uint64_t blend_evals;     /* FGS_RENDER_COUNT: pixel-Gaussian evaluations (pixels not stopped) */
    uint64_t blend_hits;      /* FGS_RENDER_COUNT: evaluations that reached alpha / T (exp taken) */
    uint64_t blend_active;    /* FGS_RENDER_COUNT: lockstep steps where some pixel reached it */
    uint64_t filter_in_frustum;  /* FGS_RENDER_COUNT: nodes whose centre passes the frustum test */
    uint64_t filter_cov_nodes;   /* FGS_RENDER_COUNT: in-frustum internal nodes, the only ones whose
                                    covariance the R&L filter must read (a leaf passes on the
                                    frustum test alone) */
    uint64_t filter_chunks_read; /* FGS_RENDER_COUNT: 128-node chunks whose centres the R&L filter
                                    read (the others lie wholly outside the frustum) */
} fgs_stats;

/* Library version (FGS_VERSION). */
int fgs_version(void);

/* Create a context on CUDA device `device` with default parameters
 * (tau_R 3, 16x16 tiles, black background, 32 Mi pairs).  *out receives the
 * handle.  Errors: FGS_ERR_ARG, FGS_ERR_CUDA, FGS_ERR_NOMEM. */
int fgs_create(fgs_ctx** out, int device);

/* Free every device buffer of the context and the context itself.  Waits for
 * work of the context to finish.  NULL is accepted. */
int fgs_destroy(fgs_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  The string
 * is owned by the context and valid until its next call. */
const char* fgs_last_error(const fgs_ctx* ctx);

/* Set render parameters.  A non-zero pair_capacity reallocates the pair
 * buffers to exactly that many pairs.
 * Errors: FGS_ERR_ARG (tile not a power of two or not 256 pixels, NaN). */
int fgs_set_params(fgs_ctx* ctx, const fgs_params* p);

/* Validate a tree (host arrays, layout above) without any device work:
 * one root, parent ids in range and acyclic, is_leaf equals "has no
 * children", AP rows equal the parent chain, depth covers the longest path,
 * finite attributes, opacity in (0, 1].  On failure writes a message into
 * msg (msg_len bytes, may be NULL).  Returns FGS_OK, FGS_ERR_ARG or
 * FGS_ERR_TREE.  Callable without a GPU. */
int fgs_validate_tree(const fgs_tree* tree, char* msg, size_t msg_len);

/* Validate (as fgs_validate_tree) and upload a tree (host arrays).  Validation: one
 * root, parent ids in range and acyclic, is_leaf equals "has no children",
 * AP rows equal the parent chain, depth covers the longest path, finite
 * attributes.  Replaces a previously loaded tree.  Errors: FGS_ERR_ARG,
 * FGS_ERR_TREE, FGS_ERR_NOMEM, FGS_ERR_CUDA. */
int fgs_load_tree(fgs_ctx* ctx, const fgs_tree* tree);

/* Set the camera used by the next frame calls (copied; host struct).  Grows
 * the tile buffers if the image has more tiles.  Errors: FGS_ERR_ARG for
 * non-finite values, width/height outside 1..16384, tan_half <= 0, or more
 * than 65,536 tiles with the current tile shape (the (tile | depth) keys hold
 * 16 tile bits: 6 digit passes). */
int fgs_set_camera(fgs_ctx* ctx, const fgs_camera* cam);

/* Footprint mode for the next frames (§3.3): FGS_SHRINK_OFF (3 sigma) or
 * FGS_SHRINK_ON with threshold tau and ln_tau = ln(tau) (both supplied by
 * the caller, typically from fgs_calibrate_gtc(), so the CUDA path and any
 * checker use the same bits).  Errors: FGS_ERR_ARG. */
int fgs_set_shrink(fgs_ctx* ctx, int mode, float tau, float ln_tau);

/* Run the filter only (§3.2): R&L + Ancestor filters and compaction.
 * sel_out receives the selected node ids in ascending order (up to cap of
 * them), *M_out the count M (may exceed cap; then only cap ids are
 * written and FGS_ERR_CAPACITY is returned).  out_is_device: 1 if sel_out
 * and M_out are device pointers (asynchronous), 0 for host pointers
 * (synchronising). */
int fgs_filter(fgs_ctx* ctx, void* stream, uint32_t* sel_out, uint32_t cap, uint32_t* M_out,
               int out_is_device);

/* Comparison baseline of §3.2 (Eq. 3): the serial level-by-level selection
 * that the traversal-free filter replaces.  From the root, one kernel per tree
 * level evaluates R&L for the current frontier; a node that passes is
 * selected, otherwise its children form the next frontier.  The host reads the
 * frontier size after every level (one launch and one synchronisation per
 * level).  Returns the same selection as fgs_filter (ascending ids, up to cap;
 * *M_out = M), and the number of levels visited in *levels_out (may be NULL).
 * Synchronising (host round trip per level) whatever out_is_device says.
 * Errors as fgs_filter. */
int fgs_filter_levelwise(fgs_ctx* ctx, void* stream, uint32_t* sel_out, uint32_t cap,
                         uint32_t* M_out, int out_is_device, uint32_t* levels_out);

/* Render one frame of the current camera: filter, project, shrink, count the
 * pairs per tile, tile ranges, scatter the pairs into per-tile buckets, sort
 * each bucket, blend.  rgb_out: float [3][H][W] planar colour
 * C + T * bg; T_out: float [H][W] final transmittance (may be NULL).
 * out_is_device selects device (asynchronous) or host (synchronising)
 * outputs; with FGS_RENDER_ASYNC host outputs do not synchronise either: the
 * call returns once the frame and its copy are enqueued, the copy (a pinned
 * host buffer lets it overlap the next frame's kernels) runs on the context's
 * copy stream, latched device errors are reported by fgs_sync, and the host
 * buffers must not be read or reused before fgs_sync returns.  The third
 * pipelined frame's blend waits on the device for the first one's copy.
 * flags: FGS_RENDER_STATS fills st->n_selected / n_pairs /
 * device_status (synchronising); FGS_RENDER_STAGE_EVENTS records stage events
 * into the next slot of a 256-slot ring (see fgs_stage_times).  st may be
 * NULL.  Errors: FGS_ERR_STATE (no tree or camera), FGS_ERR_ARG,
 * FGS_ERR_CUDA, and latched device errors when synchronising. */
int fgs_render(fgs_ctx* ctx, void* stream, float* rgb_out, float* T_out, int out_is_device,
               uint32_t flags, fgs_stats* st);

/* Per-stage durations (ms, CUDA events) of the frame recorded in ring slot
 * `slot` (0..255, in call order modulo 256): FGS_N_STAGES values.  Waits for
 * those events.  Errors: FGS_ERR_ARG (slot never recorded). */
int fgs_stage_times(fgs_ctx* ctx, int slot, float* ms_out);

/* Number of frames recorded with FGS_RENDER_STAGE_EVENTS so far. */
int fgs_stage_count(const fgs_ctx* ctx, uint64_t* count_out);

/* Copy the sorted Gaussian-tile pairs of the last frame: keys
 * (tile << 32 | depth bits) and values (rank of the Gaussian in the
 * selection).  At most cap pairs; *n_out = N_P.  Synchronising for host
 * outputs.  Errors: FGS_ERR_STATE (no frame yet), FGS_ERR_CAPACITY. */
int fgs_get_pairs(fgs_ctx* ctx, void* stream, uint64_t* keys_out, uint32_t* vals_out,
                  uint64_t cap, uint64_t* n_out, int out_is_device);

/* Copy the projected splats of the last frame: float [M][12] rows of
 * u, v, conic A, B, C, ln-threshold, alpha_0, depth, r, g, b, footprint
 * radius (0 when the Gaussian is dropped by shrinking or has a singular
 * conic; conic 0 in the latter case), in selection order.  r, g, b are
 * evaluated only for Gaussians that emit at least one pair (0 otherwise:
 * no pixel reads them).
 * *M_out = M.  Errors as fgs_get_pairs. */
int fgs_get_splats(fgs_ctx* ctx, void* stream, float* out, uint32_t cap, uint32_t* M_out,
                   int out_is_device);

/* Calibration pre-render of the current camera with the 3-sigma footprint
 * (§3.3): KPC of every sorted pair (Eq. 5), GTC per tile (Eq. 6, NaN for
 * tiles without pairs) and the view average G_v (Eq. 7) over tiles that have
 * pairs.  kpc_out (float [N_P], may be NULL, at most kpc_cap values) and
 * G_out (float [tiles], may be NULL) are host or device per out_is_device;
 * gbar_out is a host double.  Synchronising.  Leaves the shrink mode
 * unchanged. */
int fgs_calibrate_view(fgs_ctx* ctx, void* stream, double* gbar_out, float* kpc_out,
                       uint64_t kpc_cap, float* G_out, int out_is_device);

/* As fgs_calibrate_view, but under the context's current footprint mode
 * (3-sigma, or shrunk to tau when shrinking is on): the KPC of every pair the
 * shrunk frame emits, the per-tile GTC and the view average.  Serves the study
 * of redundant pairs (§3.3: pairs whose KPC is near zero) before and after
 * shrinking.  Same arguments, outputs and errors as fgs_calibrate_view. */
int fgs_kpc_view(fgs_ctx* ctx, void* stream, double* gbar_out, float* kpc_out, uint64_t kpc_cap,
                 float* G_out, int out_is_device);

/* Scene calibration (§3.3, Eq. 8): pre-render n_views cameras (host array),
 * G = mean of their G_v, tau = lambda_G / G, ln_tau = ln lambda_G - ln G
 * (float64, rounded once).  gbar_views_out (host, n_views doubles) may be
 * NULL.  Leaves the last view as the current camera.  Does NOT switch
 * shrinking on: pass tau / ln_tau to fgs_set_shrink(). */
int fgs_calibrate_gtc(fgs_ctx* ctx, void* stream, const fgs_camera* views, int n_views,
                      float lambda_G, double* gbar_views_out, float* tau_out, float* ln_tau_out);

/* Diagnostic: evaluate the blend's binary32 exp (Cody-Waite reduction,
 * degree-7 Taylor polynomial, fused multiply-adds in a fixed order) on n device
 * floats x -> y (device pointers) on `stream`.  Asynchronous.  Errors:
 * FGS_ERR_ARG, FGS_ERR_CUDA. */
int fgs_eval_exp(const float* x, float* y, uint64_t n, void* stream);

/* Diagnostic of the failure detection (no counterpart in the paper): launches
 * one warp that waits, through the decoupled look-back wait the compaction
 * uses, on a predecessor entry that nothing publishes (a tag no frame uses).
 * The wait gives up after 4096 empty rounds (milliseconds; the render's waits
 * allow 2^24) and latches the device status FGS_ERR_TIMEOUT, as a wait that
 * runs out in a frame does; the kernel then returns.  The call clears any
 * earlier status, synchronises `stream`, reads the status, clears it again and
 * returns it: FGS_ERR_TIMEOUT (with *site_out = 0x7F0, the probe's site code)
 * is the expected result; FGS_OK would mean the wait ended without its bound.
 * The context stays usable.  Needs a loaded tree (its look-back buffer); do not
 * overlap it with a render of the same context on another stream.  Errors:
 * FGS_ERR_ARG, FGS_ERR_STATE, FGS_ERR_CUDA. */
int fgs_probe_wait_timeout(fgs_ctx* ctx, void* stream, uint32_t* site_out);

/* Allocation-free compaction of selection bits (no counterpart in the paper:
 * a service for callers that cannot allocate device memory, e.g. a host
 * application that owns every allocation, code running during CUDA stream
 * capture, or a real-time loop that may not allocate after start-up).
 * Writes the indices of the set bits of selbits[n_words] (bit b of word w is
 * index 32 w + b) in ascending order to ids_out, and their number to
 * count_out[0] (0xFFFFFFFF if a bounded device wait timed out).  All pointers
 * are device pointers; ids_out must hold every set bit (at most 32 * n_words
 * indices).  Runs the render path's compaction kernel, but its scratch (one
 * 64-bit look-back word per 32K-index tile, 512 KiB, and a 256-byte state
 * block: 524,544 bytes) is a static device array of the library,
 * so the call allocates nothing.  Limit: n_words <= 2^26
 * (2^31 indices); larger inputs return FGS_ERR_ARG before any launch.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (other streams, other threads) race;
 * serialise them.  Asynchronous on `stream` (the current device's).  Errors:
 * FGS_ERR_ARG, FGS_ERR_CUDA. */
int fgs_compact_selection_noalloc(const uint32_t* selbits, uint64_t n_words, uint32_t* ids_out,
                                  uint32_t* count_out, void* stream);

/* Batched multi-view form (next form beside §3.2-§3.3's single view: many
 * views of uneven resolution per call).  Set-up for n_views (1..64) cameras
 * (host array): tile_shapes (may be NULL = the context's tile and blend warp
 * shape) holds {tile_w, tile_h, blend_warp_w} per view; sel_capacity / pair_capacity bound the selected
 * entries and Gaussian-tile pairs of the whole batch (0 = defaults: views x
 * nodes up to 64 Mi entries, 128 Mi pairs).  Allocates the batch buffers.
 * The batch keeps the context's tau_R, background and shrink mode as they are
 * at each fgs_render_batch call.  Errors: FGS_ERR_ARG, FGS_ERR_STATE (no
 * tree), FGS_ERR_NOMEM. */
int fgs_batch_setup(fgs_ctx* ctx, const fgs_camera* views, int n_views, const int32_t* tile_shapes,
                    uint64_t sel_capacity, uint64_t pair_capacity);

/* Replace the batch's cameras (same count and resolutions; host array). */
int fgs_batch_set_cameras(fgs_ctx* ctx, const fgs_camera* views, int n_views);

/* Pixel offset of every view's image in the batch outputs: offsets_out[v]
 * (n_views + 1 values, host).  View v's colour planes start at
 * rgb_out + 3 * offsets_out[v] ([3][H_v][W_v]) and its transmittance at
 * T_out + offsets_out[v]; offsets_out[n_views] is the total pixel count. */
int fgs_batch_image_offsets(const fgs_ctx* ctx, uint64_t* offsets_out);

/* Render every view of the batch with one pass of the kernels over all views:
 * multi-view R&L and Ancestor filters (each node and ancestor path read once
 * for all views), one compaction, one projection with pairs counted into
 * global tile ids (a view's first tile + the tile), one tile scan, key scatter
 * and per-tile sort over every view's tiles, one blend launch over all views'
 * tiles.  Per view the result equals fgs_render with the same camera
 * and tile shape.  rgb_out / T_out are DEVICE buffers of 3 * total and total
 * pixels (see fgs_batch_image_offsets); T_out may be NULL.  flags:
 * FGS_BATCH_GRAPH replays a CUDA graph captured on first use for these output
 * pointers (re-captured when they change); FGS_RENDER_STATS synchronises and
 * fills st (n_selected, n_pairs over the batch).  Asynchronous otherwise.
 * Errors: FGS_ERR_STATE (no set-up), FGS_ERR_CAPACITY (with STATS), CUDA. */
int fgs_render_batch(fgs_ctx* ctx, void* stream, float* rgb_out, float* T_out, uint32_t flags,
                     fgs_stats* st);

/* Copy the intermediate results of the last fgs_render_batch, so that each
 * view can be checked against the single-view path: the selected entries
 * (entry = view * node_stride + node, ascending: view, then node id), their
 * projected splats (float [M][12], fields as fgs_get_splats, in entry order)
 * and the sorted Gaussian-tile pairs of the whole batch (keys
 * (global tile << 32 | depth bits), values = index of the entry in the
 * selected list).  View v's global tiles are [tile_base_out[v],
 * tile_base_out[v + 1]) (n_views + 1 values); its tile t (row-major in its own
 * tile grid) has the global id tile_base_out[v] + t.  All outputs are HOST
 * buffers; any of the arrays may be NULL; at most sel_cap entries / splat rows
 * and pair_cap pairs are copied; *M_out and *NP_out receive the batch totals.
 * With every array NULL the call only reports the totals (a size query).
 * Synchronising.  Errors: FGS_ERR_ARG, FGS_ERR_STATE (no batch rendered since
 * the set-up or the last tree load), FGS_ERR_CAPACITY (a total above the cap
 * of an array that was given, or a capacity error latched by the render),
 * FGS_ERR_TIMEOUT, FGS_ERR_CUDA. */
int fgs_batch_get_frame(fgs_ctx* ctx, void* stream, uint32_t* entries_out, float* splat_out,
                        uint64_t sel_cap, uint64_t* M_out, uint64_t* keys_out, uint32_t* vals_out,
                        uint64_t pair_cap, uint64_t* NP_out, uint32_t* node_stride_out,
                        uint32_t* tile_base_out);

/* ---- differentiable form -----------------------------------------------
 * The render as a function of per-node Gaussian parameters, in the 3D Gaussian
 * splatting parametrisation the method builds on (§3.1), and its gradient.
 * The selection (§3.2 cut), the Gaussian-tile pairs and every skip / stop /
 * clamp decision of blending (Eq. 2) are held fixed: the gradient is the one
 * of the image with those discrete choices frozen, as when a cut is trained.
 *
 * Parameter arrays are DEVICE pointers on the context's device, n = n_nodes of
 * the loaded tree, float32, row-major:
 *   mu[3][n]         centre
 *   log_scale[3][n]  Sigma = R diag(e^{2 s}) R^T
 *   quat[4][n]       (w, x, y, z), any non-zero norm; R = R(q / |q|)
 *   logit[n]         alpha0 = 1 / (1 + e^{-l}), l clamped to [-80, 80]
 *                    (zero gradient outside)
 *   sh[n][K][3]      SH coefficients, K = (sh_degree + 1)^2;
 *                    colour = max(0, 1/2 + sum_k Y_k(d) c_k), d the unit
 *                    direction from the camera centre
 * The caller owns them; the library reads (and for grads writes) them during
 * the call's kernels only. */
typedef struct fgs_gauss_params {
    const float* mu;
    const float* log_scale;
    const float* quat;
    const float* logit;
    const float* sh;
} fgs_gauss_params;

typedef struct fgs_gauss_grads {
    float* mu;
    float* log_scale;
    float* quat;
    float* logit;
    float* sh;
} fgs_gauss_grads;

#define FGS_BACKWARD_ACCUMULATE 1u  /* add into the gradient arrays instead of overwriting */

/* Recompute the loaded tree's attributes from parameters: mean, Sigma,
 * alpha0, ln alpha0 (the binary32 values the filter, projection and blending
 * decide on, in one fixed operation order: Sigma_ij = ((R_i0 s_0) R_j0 +
 * (R_i1 s_1) R_j1) + (R_i2 s_2) R_j2 with s_k = exp(2 log_scale_k) and the
 * exp / ln of the library's own binary32 routines) and SH.  The tree
 * structure (parents, leaves, ancestor paths) is unchanged.  Asynchronous on
 * `stream`.  Errors: FGS_ERR_STATE (no tree), FGS_ERR_ARG (NULL or non-device
 * pointer), FGS_ERR_CUDA. */
int fgs_update_params(fgs_ctx* ctx, void* stream, const fgs_gauss_params* p);

/* Gradient of L = sum over pixels and channels of dL_drgb * rgb for the last
 * fgs_render of this context (same camera, parameters as passed to the last
 * fgs_update_params).  dL_drgb: DEVICE [3][H][W] (the layout of fgs_render's
 * rgb_out).  p: the parameters of that render; g: gradient arrays of the same
 * shapes (device).  Without FGS_BACKWARD_ACCUMULATE every entry of g is
 * written (zero for nodes outside the cut); with it, the selected nodes'
 * gradients are added.  Two kernels: a per-tile blend backward that
 * recomputes each pixel's final transmittance and stop position by a
 * front-to-back walk over its tile (or reads them, if the render used
 * FGS_RENDER_KEEP) and then walks the tile back to front, recovering T before
 * each Gaussian as T / (1 - alpha); and a per-Gaussian chain rule through the
 * conic, the EWA Jacobian, Sigma(q, s), the sigmoid and the SH basis.
 * Asynchronous on `stream`.  Errors: FGS_ERR_STATE (no rendered frame since
 * the last change of tree, camera, parameters or settings), FGS_ERR_ARG,
 * FGS_ERR_NOMEM, FGS_ERR_CUDA. */
int fgs_backward(fgs_ctx* ctx, void* stream, const float* dL_drgb, const fgs_gauss_params* p,
                 const fgs_gauss_grads* g, uint32_t flags);

/* Wait for the stream and return any latched device status, then clear it. */
int fgs_sync(fgs_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FILTERGS_H */
