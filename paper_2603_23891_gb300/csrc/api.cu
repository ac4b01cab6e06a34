// C ABI of the FilterGS render path: context, tree upload and validation,
// camera / parameter state, frame orchestration on the caller's stream.
#include "filtergs.h"
#include "fgs_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace fgs;

namespace {

constexpr int kEventSlots = 256;
constexpr uint64_t kDefaultPairCap = 32ull << 20;
constexpr uint64_t kMaxPairCap = (1ull << 31) - 64;
constexpr int kMaxTiles = 1 << 16;

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct fgs_ctx {
    int device = 0;
    int sms = 1;
    std::string err;
    fgs_params params{};
    // occupancy (resident blocks per SM)
    int occ_pred = 1, occ_anc = 1, occ_compact = 1, occ_proj = 1, occ_scatter = 1, occ_segsort = 1, occ_scan = 1;
    // tree
    bool has_tree = false;
    DevTree tree{};
    void* tree_mem = nullptr;
    // children (CSR) for the level-wise baseline, and its frontiers
    uint32_t root = 0;
    uint32_t* child_start = nullptr;
    uint32_t* children = nullptr;
    uint32_t* frontier0 = nullptr;
    uint32_t* frontier1 = nullptr;
    uint32_t* d_counter = nullptr;
    uint32_t* h_counter = nullptr;   // pinned
    // camera / shrink
    bool has_cam = false;
    fgs_camera cam{};
    int shrink = FGS_SHRINK_OFF;
    float tau = 0.0f, ln_tau = -INFINITY;
    // node-sized frame buffers
    size_t node_cap = 0;
    uint32_t* pbits = nullptr;
    uint32_t* selbits = nullptr;
    uint32_t* sel = nullptr;
    float* splat = nullptr;
    unsigned long long* lb_compact = nullptr;
    uint32_t* sel_cnt = nullptr;    // selected nodes per 256-word tile (the Ancestor filter's counts)
    uint4* foot = nullptr;          // per selected Gaussian: rect, pair count, depth bits
    // pair-sized buffers
    uint64_t pair_cap = 0;
    unsigned long long* keys0 = nullptr;
    unsigned long long* keys1 = nullptr;
    uint32_t* vals0 = nullptr;
    uint32_t* vals1 = nullptr;
    float* kpc = nullptr;
    // tile-sized buffers
    size_t tile_cap = 0;
    uint2* ranges = nullptr;
    uint32_t* tile_cnt = nullptr;   // pairs per tile, then the tile's scatter cursor
    uint32_t* large = nullptr;      // tiles whose pairs one block sorts
    unsigned long long* lb_scan = nullptr;   // the tile scan's look-back entries
    float* G = nullptr;
    // image staging for host outputs: rgb planes + T
    size_t img_cap = 0;
    float* img = nullptr;
    uint2* keep = nullptr;          // per pixel: final T bits, stop position (for the backward)
    // pipelined host outputs (FGS_RENDER_ASYNC): two device images, each frame's
    // copy to the host on copy_stream; ev_blend[i] marks image i written,
    // ev_copied[i] its copy done (the frame after next waits for it)
    size_t ring_cap = 0;
    float* ring[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_blend[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    bool ring_busy[2] = {false, false};
    int ring_next = 0;
    // frame state
    FrameState* st = nullptr;
    FrameState* st_host = nullptr;
    // stage events
    bool ev_ready = false;
    cudaEvent_t ev[kEventSlots][kStages + 1];
    uint64_t ev_count = 0;
    // differentiable form: per selected Gaussian splat gradients
    float* gsplat = nullptr;
    size_t gsplat_rows = 0;
    // last frame
    bool have_frame = false;
    bool frame_rendered = false;    // the last frame came from fgs_render (not a calibration)
    bool frame_kept = false;        // ... with FGS_RENDER_KEEP
    // batched multi-view state
    struct Batch {
        int V = 0;
        std::vector<fgs_camera> cams;
        std::vector<int32_t> tile_w, tile_h, warp_w;
        std::vector<uint32_t> tile_base;          // V + 1
        std::vector<unsigned long long> img_off;  // V + 1 (pixels)
        uint32_t total_tiles = 0;
        uint64_t sel_cap = 0, pair_cap = 0;
        DevCamera* d_cams = nullptr;
        DevCamera* h_cams = nullptr;              // pinned staging
        uint32_t* d_tile_base = nullptr;
        unsigned long long* d_img_off = nullptr;
        uint32_t *pbits = nullptr, *selbits = nullptr, *sel = nullptr;
        float* splat = nullptr;
        uint4* foot = nullptr;
        unsigned long long *items = nullptr, *keys = nullptr, *lb_compact = nullptr, *lb_scan = nullptr;
        uint32_t* vals = nullptr;
        uint2* ranges = nullptr;
        uint32_t *tile_cnt = nullptr, *large = nullptr;
        FrameState* st = nullptr;
        cudaGraphExec_t graph = nullptr;
        float* graph_rgb = nullptr;
        float* graph_T = nullptr;
        bool have_frame = false;                  // a batch has been rendered since the set-up
    } batch;
};

namespace {

bool finite_all(const float* p, size_t n);

int fail(fgs_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define FGS_CUDA(ctx, expr)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? FGS_ERR_NOMEM : FGS_ERR_CUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

void free_ptr(void* p)
{
    if (p) cudaFree(p);
}

int grow(fgs_ctx* c, void** p, size_t bytes)
{
    free_ptr(*p);
    *p = nullptr;
    if (bytes == 0) return FGS_OK;
    FGS_CUDA(c, cudaMalloc(p, bytes));
    FGS_CUDA(c, cudaMemset(*p, 0, bytes));
    return FGS_OK;
}

// Pair buffers sized exactly for `cap` pairs (reallocated when it changes).
int ensure_pairs(fgs_ctx* c, uint64_t cap)
{
    if (cap == c->pair_cap) return FGS_OK;
    int r;
    const size_t n = (size_t)cap + 8;   // TMA reads an aligned superset of a slice
    if ((r = grow(c, (void**)&c->keys0, n * 8))) return r;
    if ((r = grow(c, (void**)&c->keys1, n * 8))) return r;
    if ((r = grow(c, (void**)&c->vals0, n * 4))) return r;
    if ((r = grow(c, (void**)&c->vals1, n * 4))) return r;
    if ((r = grow(c, (void**)&c->kpc, n * 4))) return r;
    c->pair_cap = cap;
    c->have_frame = false;
    return FGS_OK;
}

int ensure_nodes(fgs_ctx* c, size_t n_pad)
{
    if (n_pad <= c->node_cap) return FGS_OK;
    int r;
    if ((r = grow(c, (void**)&c->pbits, n_pad / 32 * 4))) return r;
    if ((r = grow(c, (void**)&c->selbits, n_pad / 32 * 4))) return r;
    if ((r = grow(c, (void**)&c->sel, n_pad * 4))) return r;
    if ((r = grow(c, (void**)&c->splat, n_pad * kSplatStride * 4))) return r;
    if ((r = grow(c, (void**)&c->lb_compact, (n_pad / 32 / kCompactWords + 2) * 8))) return r;
    if ((r = grow(c, (void**)&c->sel_cnt, (n_pad / 32 / kSelTileWords + 2) * 4))) return r;
    if ((r = grow(c, (void**)&c->foot, n_pad * sizeof(uint4)))) return r;
    c->node_cap = n_pad;
    return FGS_OK;
}

// The two device images of pipelined host outputs (rgb planes + T, `pixels`
// each), the copy stream and its events, created on first use.  Growing the
// images first waits for the copies that read them.
int ensure_ring(fgs_ctx* c, size_t pixels)
{
    int r;
    if (!c->copy_stream) {
        FGS_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            FGS_CUDA(c, cudaEventCreateWithFlags(&c->ev_blend[i], cudaEventDisableTiming));
            FGS_CUDA(c, cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming));
        }
    }
    if (pixels > c->ring_cap) {
        FGS_CUDA(c, cudaStreamSynchronize(c->copy_stream));
        for (int i = 0; i < 2; ++i)
            if ((r = grow(c, (void**)&c->ring[i], pixels * 4 * 4))) return r;
        c->ring_busy[0] = c->ring_busy[1] = false;
        c->ring_cap = pixels;
    }
    return FGS_OK;
}

int ensure_tiles(fgs_ctx* c, size_t tiles, size_t pixels)
{
    int r;
    if (tiles > c->tile_cap) {
        if ((r = grow(c, (void**)&c->ranges, tiles * sizeof(uint2)))) return r;
        if ((r = grow(c, (void**)&c->tile_cnt, tiles * 4))) return r;
        if ((r = grow(c, (void**)&c->large, tiles * 4))) return r;
        if ((r = grow(c, (void**)&c->lb_scan, tile_scan_lookback_entries(tiles) * 8))) return r;
        if ((r = grow(c, (void**)&c->G, tiles * 4))) return r;
        c->tile_cap = tiles;
    }
    if (pixels > c->img_cap) {
        if ((r = grow(c, (void**)&c->img, pixels * 4 * 4))) return r;
        if ((r = grow(c, (void**)&c->keep, pixels * sizeof(uint2)))) return r;
        c->img_cap = pixels;
    }
    return FGS_OK;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v)
{
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
}

DevCamera make_devcam(const fgs_ctx* c, bool force_shrink_off)
{
    DevCamera d{};
    std::memcpy(d.R, c->cam.R, sizeof d.R);
    std::memcpy(d.t, c->cam.t, sizeof d.t);
    d.fx = c->cam.fx;
    d.fy = c->cam.fy;
    d.cx = c->cam.cx;
    d.cy = c->cam.cy;
    d.tan_half_x = c->cam.tan_half_x;
    d.tan_half_y = c->cam.tan_half_y;
    std::memcpy(d.campos, c->cam.campos, sizeof d.campos);
    d.width = c->cam.width;
    d.height = c->cam.height;
    d.tile_w = c->params.tile_w;
    d.tile_h = c->params.tile_h;
    d.tile_shift_x = ilog2(d.tile_w);
    d.tile_shift_y = ilog2(d.tile_h);
    d.tiles_x = (d.width + d.tile_w - 1) / d.tile_w;
    d.tiles_y = (d.height + d.tile_h - 1) / d.tile_h;
    d.tau_R = c->params.tau_R;
    d.shrink = force_shrink_off ? 0 : c->shrink;
    d.tau = c->tau;
    d.ln_tau = c->ln_tau;
    std::memcpy(d.bg, c->params.bg, sizeof d.bg);
    d.warp_shift = c->params.blend_warp_w == 4 ? 2 : 3;
    return d;
}

DevCamera make_devcam_for(const fgs_ctx* c, const fgs_camera& cam, int tile_w, int tile_h, int warp_w)
{
    DevCamera d{};
    std::memcpy(d.R, cam.R, sizeof d.R);
    std::memcpy(d.t, cam.t, sizeof d.t);
    d.fx = cam.fx;
    d.fy = cam.fy;
    d.cx = cam.cx;
    d.cy = cam.cy;
    d.tan_half_x = cam.tan_half_x;
    d.tan_half_y = cam.tan_half_y;
    std::memcpy(d.campos, cam.campos, sizeof d.campos);
    d.width = cam.width;
    d.height = cam.height;
    d.tile_w = tile_w;
    d.tile_h = tile_h;
    d.tile_shift_x = ilog2(tile_w);
    d.tile_shift_y = ilog2(tile_h);
    d.tiles_x = (d.width + tile_w - 1) / tile_w;
    d.tiles_y = (d.height + tile_h - 1) / tile_h;
    d.tau_R = c->params.tau_R;
    d.shrink = c->shrink;
    d.tau = c->tau;
    d.ln_tau = c->ln_tau;
    std::memcpy(d.bg, c->params.bg, sizeof d.bg);
    d.warp_shift = warp_w == 4 ? 2 : 3;
    return d;
}

bool valid_camera(const fgs_camera* cam)
{
    return finite_all(cam->R, 9) && finite_all(cam->t, 3) && finite_all(cam->campos, 3) &&
           std::isfinite(cam->fx) && std::isfinite(cam->fy) && std::isfinite(cam->cx) &&
           std::isfinite(cam->cy) && cam->fx > 0 && cam->fy > 0 && cam->tan_half_x > 0 &&
           cam->tan_half_y > 0 && std::isfinite(cam->tan_half_x) && std::isfinite(cam->tan_half_y) &&
           cam->width >= 1 && cam->height >= 1 && cam->width <= 16384 && cam->height <= 16384;
}

// Counted tiles (kSelTileWords words each) of the loaded tree's selection bits.
size_t n_sel_tiles(const fgs_ctx* c) { return (c->tree.n_pad / 32 + kSelTileWords - 1) / kSelTileWords; }

int check_ready(fgs_ctx* c)
{
    if (!c) return FGS_ERR_ARG;
    if (!c->has_tree) return fail(c, FGS_ERR_STATE, "no tree loaded");
    if (!c->has_cam) return fail(c, FGS_ERR_STATE, "no camera set");
    return FGS_OK;
}

// Enqueue the frame up to the sorted pair list and its tile ranges.  Returns
// the number of kernel launches.  Stage events (if ev): filter R&L | ancestor
// filter + compaction | projection + pair counts | tile ranges | key scatter |
// per-tile sort; the caller records the blend's end.
int enqueue_front(fgs_ctx* c, const DevCamera& dc, cudaStream_t s, cudaEvent_t* ev, bool count = false)
{
    const uint32_t tiles = (uint32_t)(dc.tiles_x * dc.tiles_y);
    if (ev) cudaEventRecord(ev[0], s);
    launch_frame_begin(c->st, c->tile_cnt, (int)tiles, c->sel_cnt, (int)n_sel_tiles(c), s);
    launch_filter_pred(c->tree, dc, c->pbits, count ? c->st : nullptr, c->sms * c->occ_pred, s);
    if (ev) cudaEventRecord(ev[1], s);
    launch_filter_anc(c->tree, c->pbits, c->selbits, c->sel_cnt, c->sms * c->occ_anc, s);
    launch_compact_counted(c->selbits, c->tree.n_pad / 32, c->sel, c->tree.n_pad, c->sel_cnt, c->st, s);
    if (ev) cudaEventRecord(ev[2], s);
    launch_project(c->tree, dc, c->sel, c->splat, c->foot, c->tile_cnt, c->st, c->sms * c->occ_proj, s);
    if (ev) cudaEventRecord(ev[3], s);
    launch_tile_scan(c->tile_cnt, c->ranges, tiles, c->large, c->pair_cap, c->lb_scan, c->st, c->sms * c->occ_scan,
                     s);
    if (ev) cudaEventRecord(ev[4], s);
    launch_scatter(dc, c->foot, c->tile_cnt, c->keys0, c->pair_cap, c->st, c->sms * c->occ_scatter, s);
    if (ev) cudaEventRecord(ev[5], s);
    launch_segsort(c->ranges, tiles, c->large, c->keys0, c->keys1, c->vals1, c->st,
                   c->sms * c->occ_segsort, s);
    if (ev) cudaEventRecord(ev[6], s);
    return 8;
}

int read_state(fgs_ctx* c, cudaStream_t s)
{
    FGS_CUDA(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(FrameState), cudaMemcpyDeviceToHost, s));
    FGS_CUDA(c, cudaStreamSynchronize(s));
    return FGS_OK;
}

int latched_status(fgs_ctx* c)
{
    const int st = c->st_host->status;
    if (st == 0) return FGS_OK;
    if (st == kErrCapacity)
        return fail(c, FGS_ERR_CAPACITY, "pair capacity %llu exceeded (N_P = %llu)",
                    (unsigned long long)c->pair_cap, (unsigned long long)c->st_host->n_pairs);
    if (st == kErrTimeout)
        return fail(c, FGS_ERR_TIMEOUT, "device spin-wait timed out (site 0x%x)", c->st_host->status_info);
    return fail(c, FGS_ERR_CUDA, "device status %d", st);
}

int clear_status(fgs_ctx* c, cudaStream_t s)
{
    FGS_CUDA(c, cudaMemsetAsync(&c->st->status, 0, 2 * sizeof(int32_t), s));
    return FGS_OK;
}

bool finite_all(const float* p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int fgs_version(void) { return FGS_VERSION; }

int fgs_create(fgs_ctx** out, int device)
{
    if (!out) return FGS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FGS_ERR_ARG;
    DeviceGuard g(device);
    if (!g.ok) return FGS_ERR_CUDA;
    fgs_ctx* c = new fgs_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    c->occ_pred = occ_filter_pred();
    c->occ_anc = occ_filter_anc();
    c->occ_compact = occ_compact();
    c->occ_proj = occ_project();
    c->occ_scatter = occ_scatter();
    c->occ_segsort = occ_segsort();
    c->occ_scan = occ_tile_scan();
    c->params.tau_R = 3.0f;
    c->params.tile_w = 16;
    c->params.tile_h = 16;
    c->params.blend_warp_w = 8;
    c->params.bg[0] = c->params.bg[1] = c->params.bg[2] = 0.0f;
    c->params.pair_capacity = kDefaultPairCap;
    int r = FGS_OK;
    if (cudaMalloc((void**)&c->st, sizeof(FrameState)) != cudaSuccess ||
        cudaMemset(c->st, 0, sizeof(FrameState)) != cudaSuccess ||
        cudaMallocHost((void**)&c->st_host, sizeof(FrameState)) != cudaSuccess)
        r = FGS_ERR_NOMEM;
    if (r == FGS_OK) r = ensure_pairs(c, kDefaultPairCap);
    if (r != FGS_OK) {
        fgs_destroy(c);
        return r;
    }
    std::memset(c->st_host, 0, sizeof(FrameState));
    *out = c;
    return FGS_OK;
}

int fgs_destroy(fgs_ctx* c)
{
    if (!c) return FGS_OK;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    void* bufs[] = {c->child_start, c->children, c->frontier0, c->frontier1, c->d_counter,
                    c->tree_mem, c->pbits, c->selbits, c->sel, c->splat, c->lb_compact, c->sel_cnt, c->foot,
                    c->keys0, c->keys1, c->vals0, c->vals1, c->kpc, c->ranges, c->tile_cnt, c->large, c->lb_scan,
                    c->G, c->img, c->keep, c->st, c->gsplat};
    for (void* p : bufs) free_ptr(p);
    for (float* p : c->ring) free_ptr(p);
    for (int i = 0; i < 2; ++i) {
        if (c->ev_blend[i]) cudaEventDestroy(c->ev_blend[i]);
        if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    {
        auto& b = c->batch;
        void* bb[] = {b.d_cams, b.d_tile_base, b.d_img_off, b.pbits, b.selbits, b.sel, b.splat,
                      b.foot, b.items, b.keys, b.vals, b.lb_compact, b.lb_scan, b.ranges, b.tile_cnt, b.large,
                      b.st};
        for (void* p : bb) free_ptr(p);
        if (b.h_cams) cudaFreeHost(b.h_cams);
        if (b.graph) cudaGraphExecDestroy(b.graph);
    }
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->h_counter) cudaFreeHost(c->h_counter);
    if (c->ev_ready)
        for (int i = 0; i < kEventSlots; ++i)
            for (int k = 0; k <= kStages; ++k) cudaEventDestroy(c->ev[i][k]);
    delete c;
    return FGS_OK;
}

const char* fgs_last_error(const fgs_ctx* c) { return c ? c->err.c_str() : "null context"; }

int fgs_set_params(fgs_ctx* c, const fgs_params* p)
{
    if (!c || !p) return FGS_ERR_ARG;
    if (std::isnan(p->tau_R)) return fail(c, FGS_ERR_ARG, "tau_R is NaN");
    if (!is_pow2(p->tile_w) || !is_pow2(p->tile_h) || p->tile_w * p->tile_h != 256 ||
        p->tile_w < 8 || p->tile_h < 4)
        return fail(c, FGS_ERR_ARG, "tile %dx%d must be 64x4, 32x8, 16x16 or 8x32", p->tile_w,
                    p->tile_h);
    const int ww = p->blend_warp_w ? p->blend_warp_w : 8;
    if ((ww != 8 && ww != 4) || p->tile_h < 32 / ww)
        return fail(c, FGS_ERR_ARG, "blend warp width %d not supported for tile %dx%d", ww, p->tile_w,
                    p->tile_h);
    if (!finite_all(p->bg, 3)) return fail(c, FGS_ERR_ARG, "background not finite");
    if (p->pair_capacity > kMaxPairCap) return fail(c, FGS_ERR_ARG, "pair capacity too large");
    DeviceGuard g(c->device);
    c->params.tau_R = p->tau_R;
    c->params.tile_w = p->tile_w;
    c->params.tile_h = p->tile_h;
    c->params.blend_warp_w = ww;
    std::memcpy(c->params.bg, p->bg, sizeof p->bg);
    if (p->pair_capacity) {
        int r = ensure_pairs(c, p->pair_capacity);
        if (r) return r;
        c->params.pair_capacity = p->pair_capacity;
    }
    if (c->has_cam) {
        const DevCamera d = make_devcam(c, false);
        int r = ensure_tiles(c, (size_t)d.tiles_x * d.tiles_y, (size_t)d.width * d.height);
        if (r) return r;
    }
    c->have_frame = false;
    return FGS_OK;
}

int fgs_validate_tree(const fgs_tree* t, char* msg, size_t msg_len)
{
    auto bad = [&](int code, const char* fmt, ...) {
        if (msg && msg_len) {
            va_list ap;
            va_start(ap, fmt);
            vsnprintf(msg, msg_len, fmt, ap);
            va_end(ap);
        }
        return code;
    };
    if (msg && msg_len) msg[0] = 0;
    if (!t) return bad(FGS_ERR_ARG, "null tree");
    const uint64_t N = t->n_nodes;
    const uint32_t D = t->depth;
    if (N == 0 || N > (1ull << 31)) return bad(FGS_ERR_ARG, "n_nodes %llu out of range", (unsigned long long)N);
    if (t->sh_degree > 3) return bad(FGS_ERR_ARG, "sh_degree %u > 3", t->sh_degree);
    if (!t->mu || !t->cov || !t->opacity || !t->ln_opacity || !t->sh || !t->parent || !t->is_leaf ||
        (D > 0 && !t->ap))
        return bad(FGS_ERR_ARG, "null tree array");
    if (D > 64) return bad(FGS_ERR_ARG, "depth %u > 64", D);
    const int K = (int)((t->sh_degree + 1) * (t->sh_degree + 1));
    std::vector<uint8_t> has_child(N, 0);
    uint64_t roots = 0;
    for (uint64_t n = 0; n < N; ++n) {
        const int32_t p = t->parent[n];
        if (p == -1) {
            ++roots;
            continue;
        }
        if (p < 0 || (uint64_t)p >= N || (uint64_t)p == n)
            return bad(FGS_ERR_TREE, "node %llu has invalid parent %d", (unsigned long long)n, p);
        has_child[p] = 1;
    }
    if (roots != 1) return bad(FGS_ERR_TREE, "tree has %llu roots", (unsigned long long)roots);
    for (uint64_t n = 0; n < N; ++n)
        if ((t->is_leaf[n] != 0) != (has_child[n] == 0))
            return bad(FGS_ERR_TREE, "is_leaf[%llu] disagrees with the parent array", (unsigned long long)n);
    for (uint64_t n = 0; n < N; ++n) {
        int64_t a = t->parent[n];
        for (uint32_t k = 0; k < D; ++k) {
            const uint32_t expect = a >= 0 ? (uint32_t)a : kApPad;
            if (t->ap[(uint64_t)k * N + n] != expect)
                return bad(FGS_ERR_TREE, "AP[%u][%llu] = %u, parent chain gives %u", k,
                           (unsigned long long)n, t->ap[(uint64_t)k * N + n], expect);
            a = a >= 0 ? t->parent[a] : -1;
        }
        if (a != -1)
            return bad(FGS_ERR_TREE, "node %llu: ancestor chain longer than depth %u (or a cycle)",
                       (unsigned long long)n, D);
    }
    if (!finite_all(t->mu, 3 * N) || !finite_all(t->cov, 6 * N) || !finite_all(t->ln_opacity, N) ||
        !finite_all(t->sh, (size_t)N * K * 3))
        return bad(FGS_ERR_TREE, "non-finite tree attribute");
    for (uint64_t n = 0; n < N; ++n)
        if (!(t->opacity[n] > 0.0f && t->opacity[n] <= 1.0f))
            return bad(FGS_ERR_TREE, "opacity[%llu] = %g outside (0, 1]", (unsigned long long)n,
                       (double)t->opacity[n]);
    return FGS_OK;
}

int fgs_load_tree(fgs_ctx* c, const fgs_tree* t)
{
    if (!c || !t) return FGS_ERR_ARG;
    const uint64_t N = t->n_nodes;
    const uint32_t D = t->depth;
    const int K = (int)((t->sh_degree + 1) * (t->sh_degree + 1));

    {
        char msg[512];
        const int v = fgs_validate_tree(t, msg, sizeof msg);
        if (v != FGS_OK) return fail(c, v, "%s", msg);
    }

    // --- device layout ---------------------------------------------------
    DeviceGuard g(c->device);
    const size_t n_pad = align_up(N, kFilterTile);
    const uint32_t sh_stride = (uint32_t)align_up((size_t)K * 3, 4);
    const size_t sz_mu = 3 * n_pad * 4, sz_cov = 6 * n_pad * 4, sz_op = n_pad * 4;
    const size_t sz_sh = n_pad * sh_stride * 4, sz_leaf = n_pad / 32 * 4;
    const size_t sz_ap = (size_t)std::max<uint32_t>(D, 1) * n_pad * 4;
    size_t off = 0;
    const size_t o_mu = off; off = align_up(off + sz_mu, 256);
    const size_t o_cov = off; off = align_up(off + sz_cov, 256);
    const size_t o_op = off; off = align_up(off + sz_op, 256);
    const size_t o_lop = off; off = align_up(off + sz_op, 256);
    const size_t o_sh = off; off = align_up(off + sz_sh, 256);
    const size_t o_leaf = off; off = align_up(off + sz_leaf, 256);
    const size_t o_ap = off; off = align_up(off + sz_ap, 256);
    const size_t o_attr = off; off = align_up(off + n_pad * 48, 256);
    const size_t o_box = off; off = align_up(off + n_pad / 128 * 32, 256);
    const size_t total = off;

    free_ptr(c->tree_mem);
    c->tree_mem = nullptr;
    c->has_tree = false;
    c->have_frame = false;
    c->batch.have_frame = false;
    FGS_CUDA(c, cudaMalloc(&c->tree_mem, total));
    FGS_CUDA(c, cudaMemset(c->tree_mem, 0, total));
    char* base = (char*)c->tree_mem;
    for (int q = 0; q < 3; ++q)
        FGS_CUDA(c, cudaMemcpy(base + o_mu + q * n_pad * 4, t->mu + q * N, N * 4, cudaMemcpyHostToDevice));
    for (int q = 0; q < 6; ++q)
        FGS_CUDA(c, cudaMemcpy(base + o_cov + q * n_pad * 4, t->cov + q * N, N * 4, cudaMemcpyHostToDevice));
    FGS_CUDA(c, cudaMemcpy(base + o_op, t->opacity, N * 4, cudaMemcpyHostToDevice));
    FGS_CUDA(c, cudaMemcpy(base + o_lop, t->ln_opacity, N * 4, cudaMemcpyHostToDevice));
    if (sh_stride == (uint32_t)K * 3) {
        FGS_CUDA(c, cudaMemcpy(base + o_sh, t->sh, N * sh_stride * 4, cudaMemcpyHostToDevice));
    } else {
        FGS_CUDA(c, cudaMemcpy2D(base + o_sh, sh_stride * 4, t->sh, (size_t)K * 3 * 4, (size_t)K * 3 * 4,
                                 N, cudaMemcpyHostToDevice));
    }
    {
        std::vector<uint32_t> bits(n_pad / 32, 0);
        for (uint64_t n = 0; n < N; ++n)
            if (t->is_leaf[n]) bits[n >> 5] |= 1u << (n & 31);
        FGS_CUDA(c, cudaMemcpy(base + o_leaf, bits.data(), sz_leaf, cudaMemcpyHostToDevice));
    }
    if (D > 0) {
        FGS_CUDA(c, cudaMemcpy2D(base + o_ap, n_pad * 4, t->ap, N * 4, N * 4, D, cudaMemcpyHostToDevice));
    }
    {
        // node-major copy of the attributes the projection gathers per selected node
        std::vector<float> attr((size_t)N * 12, 0.0f);
        for (uint64_t n = 0; n < N; ++n) {
            float* a = attr.data() + n * 12;
            a[0] = t->mu[n];
            a[1] = t->mu[N + n];
            a[2] = t->mu[2 * N + n];
            a[3] = t->opacity[n];
            for (int q = 0; q < 4; ++q) a[4 + q] = t->cov[q * N + n];
            a[8] = t->cov[4 * N + n];
            a[9] = t->cov[5 * N + n];
            a[10] = t->ln_opacity[n];
        }
        FGS_CUDA(c, cudaMemcpy(base + o_attr, attr.data(), attr.size() * 4, cudaMemcpyHostToDevice));
    }
    DevTree& dt = c->tree;
    dt.n = (uint32_t)N;
    dt.n_pad = (uint32_t)n_pad;
    dt.depth = D;
    dt.sh_degree = t->sh_degree;
    dt.sh_stride = sh_stride;
    dt.mu = (const float*)(base + o_mu);
    dt.cov = (const float*)(base + o_cov);
    dt.opacity = (const float*)(base + o_op);
    dt.ln_opacity = (const float*)(base + o_lop);
    dt.sh = (const float*)(base + o_sh);
    dt.leaf_bits = (const uint32_t*)(base + o_leaf);
    dt.ap = (const uint32_t*)(base + o_ap);
    dt.attr = (const float4*)(base + o_attr);
    dt.cbox = (const float4*)(base + o_box);
    // the box of the centres of every 128 consecutive nodes (the R&L filter's
    // per-warp chunk)
    launch_chunk_boxes(dt, c->sms, 0);
    FGS_CUDA(c, cudaGetLastError());
    FGS_CUDA(c, cudaStreamSynchronize(0));
    int r = ensure_nodes(c, n_pad);
    if (r) return r;
    // children lists (CSR, ascending ids) for the level-wise baseline
    {
        std::vector<uint32_t> start(N + 1, 0), kids(N > 1 ? N - 1 : 1), fill;
        for (uint64_t n = 0; n < N; ++n) {
            if (t->parent[n] >= 0) start[t->parent[n] + 1]++;
            else c->root = (uint32_t)n;
        }
        for (uint64_t n = 0; n < N; ++n) start[n + 1] += start[n];
        fill.assign(start.begin(), start.end() - 1);
        for (uint64_t n = 0; n < N; ++n)
            if (t->parent[n] >= 0) kids[fill[t->parent[n]]++] = (uint32_t)n;
        if ((r = grow(c, (void**)&c->child_start, (N + 1) * 4))) return r;
        if ((r = grow(c, (void**)&c->children, kids.size() * 4))) return r;
        if ((r = grow(c, (void**)&c->frontier0, N * 4))) return r;
        if ((r = grow(c, (void**)&c->frontier1, N * 4))) return r;
        if (!c->d_counter && (r = grow(c, (void**)&c->d_counter, 16))) return r;
        if (!c->h_counter) FGS_CUDA(c, cudaMallocHost((void**)&c->h_counter, 16));
        FGS_CUDA(c, cudaMemcpy(c->child_start, start.data(), (N + 1) * 4, cudaMemcpyHostToDevice));
        FGS_CUDA(c, cudaMemcpy(c->children, kids.data(), kids.size() * 4, cudaMemcpyHostToDevice));
    }
    c->has_tree = true;
    return FGS_OK;
}

int fgs_set_camera(fgs_ctx* c, const fgs_camera* cam)
{
    if (!c || !cam) return FGS_ERR_ARG;
    if (!finite_all(cam->R, 9) || !finite_all(cam->t, 3) || !finite_all(cam->campos, 3) ||
        !std::isfinite(cam->fx) || !std::isfinite(cam->fy) || !std::isfinite(cam->cx) ||
        !std::isfinite(cam->cy) || !(cam->fx > 0) || !(cam->fy > 0) || !(cam->tan_half_x > 0) ||
        !(cam->tan_half_y > 0) || !std::isfinite(cam->tan_half_x) || !std::isfinite(cam->tan_half_y))
        return fail(c, FGS_ERR_ARG, "camera has non-finite or non-positive values");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return fail(c, FGS_ERR_ARG, "image %dx%d out of range", cam->width, cam->height);
    DeviceGuard g(c->device);
    const fgs_camera prev = c->cam;
    const bool had = c->has_cam;
    c->cam = *cam;
    const DevCamera d = make_devcam(c, false);
    const size_t tiles = (size_t)d.tiles_x * d.tiles_y;
    if (tiles > (size_t)kMaxTiles) {
        c->cam = prev;
        c->has_cam = had;
        return fail(c, FGS_ERR_ARG, "%zu tiles exceed %d", tiles, kMaxTiles);
    }
    int r = ensure_tiles(c, tiles, (size_t)d.width * d.height);
    if (r) return r;
    c->has_cam = true;
    c->have_frame = false;
    return FGS_OK;
}

int fgs_set_shrink(fgs_ctx* c, int mode, float tau, float ln_tau)
{
    if (!c) return FGS_ERR_ARG;
    if (mode == FGS_SHRINK_OFF) {
        c->shrink = mode;
        return FGS_OK;
    }
    if (mode != FGS_SHRINK_ON) return fail(c, FGS_ERR_ARG, "unknown shrink mode %d", mode);
    if (!std::isfinite(tau) || !(tau > 0) || !std::isfinite(ln_tau))
        return fail(c, FGS_ERR_ARG, "tau %g / ln_tau %g invalid", (double)tau, (double)ln_tau);
    c->shrink = mode;
    c->tau = tau;
    c->ln_tau = ln_tau;
    return FGS_OK;
}

int fgs_filter(fgs_ctx* c, void* stream, uint32_t* sel_out, uint32_t cap, uint32_t* M_out,
               int out_is_device)
{
    int r = check_ready(c);
    if (r) return r;
    if (!sel_out || !M_out) return fail(c, FGS_ERR_ARG, "null output");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const DevCamera dc = make_devcam(c, false);
    launch_frame_begin(c->st, c->tile_cnt, dc.tiles_x * dc.tiles_y, c->sel_cnt, (int)n_sel_tiles(c), s);
    launch_filter_pred(c->tree, dc, c->pbits, nullptr, c->sms * c->occ_pred, s);
    launch_filter_anc(c->tree, c->pbits, c->selbits, c->sel_cnt, c->sms * c->occ_anc, s);
    launch_compact_counted(c->selbits, c->tree.n_pad / 32, c->sel, c->tree.n_pad, c->sel_cnt, c->st, s);
    FGS_CUDA(c, cudaGetLastError());
    c->have_frame = false;
    if (out_is_device) {
        const size_t n = std::min<size_t>(cap, c->tree.n);
        if (n) FGS_CUDA(c, cudaMemcpyAsync(sel_out, c->sel, n * 4, cudaMemcpyDeviceToDevice, s));
        FGS_CUDA(c, cudaMemcpyAsync(M_out, &c->st->M, 4, cudaMemcpyDeviceToDevice, s));
        return FGS_OK;
    }
    if ((r = read_state(c, s))) return r;
    const uint32_t M = c->st_host->M;
    *M_out = M;
    const size_t n = std::min<size_t>(cap, M);
    if (n) FGS_CUDA(c, cudaMemcpy(sel_out, c->sel, n * 4, cudaMemcpyDeviceToHost));
    if ((r = latched_status(c))) {
        clear_status(c, s);
        return r;
    }
    if (M > cap) return fail(c, FGS_ERR_CAPACITY, "selection of %u exceeds cap %u", M, cap);
    return FGS_OK;
}

int fgs_filter_levelwise(fgs_ctx* c, void* stream, uint32_t* sel_out, uint32_t cap, uint32_t* M_out,
                         int out_is_device, uint32_t* levels_out)
{
    int r = check_ready(c);
    if (r) return r;
    if (!sel_out || !M_out) return fail(c, FGS_ERR_ARG, "null output");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const DevCamera dc = make_devcam(c, false);
    launch_frame_begin(c->st, c->tile_cnt, dc.tiles_x * dc.tiles_y, c->sel_cnt, (int)n_sel_tiles(c), s);
    FGS_CUDA(c, cudaMemsetAsync(c->selbits, 0, c->tree.n_pad / 32 * 4, s));
    c->h_counter[0] = c->root;
    FGS_CUDA(c, cudaMemcpyAsync(c->frontier0, c->h_counter, 4, cudaMemcpyHostToDevice, s));
    uint32_t n_front = 1, levels = 0;
    uint32_t* cur = c->frontier0;
    uint32_t* nxt = c->frontier1;
    while (n_front > 0 && levels <= c->tree.depth + 1) {
        FGS_CUDA(c, cudaMemsetAsync(c->d_counter, 0, 4, s));
        launch_levelwise_step(c->tree, dc, c->child_start, c->children, cur, n_front, nxt,
                              c->d_counter, c->selbits, s);
        FGS_CUDA(c, cudaMemcpyAsync(c->h_counter, c->d_counter, 4, cudaMemcpyDeviceToHost, s));
        FGS_CUDA(c, cudaStreamSynchronize(s));     // one synchronisation per level (Eq. 3)
        n_front = c->h_counter[0];
        std::swap(cur, nxt);
        ++levels;
    }
    launch_compact(c->selbits, c->tree.n_pad / 32, c->sel, c->tree.n_pad, c->lb_compact, c->st,
                   c->sms * c->occ_compact, s);
    FGS_CUDA(c, cudaGetLastError());
    c->have_frame = false;
    if (levels_out) *levels_out = levels;
    if (out_is_device) {
        const size_t n = std::min<size_t>(cap, c->tree.n);
        if (n) FGS_CUDA(c, cudaMemcpyAsync(sel_out, c->sel, n * 4, cudaMemcpyDeviceToDevice, s));
        FGS_CUDA(c, cudaMemcpyAsync(M_out, &c->st->M, 4, cudaMemcpyDeviceToDevice, s));
        return FGS_OK;
    }
    if ((r = read_state(c, s))) return r;
    const uint32_t M = c->st_host->M;
    *M_out = M;
    const size_t n = std::min<size_t>(cap, M);
    if (n) FGS_CUDA(c, cudaMemcpy(sel_out, c->sel, n * 4, cudaMemcpyDeviceToHost));
    if ((r = latched_status(c))) {
        clear_status(c, s);
        return r;
    }
    if (M > cap) return fail(c, FGS_ERR_CAPACITY, "selection of %u exceeds cap %u", M, cap);
    return FGS_OK;
}

int fgs_render(fgs_ctx* c, void* stream, float* rgb_out, float* T_out, int out_is_device,
               uint32_t flags, fgs_stats* st)
{
    int r = check_ready(c);
    if (r) return r;
    if (!rgb_out) return fail(c, FGS_ERR_ARG, "null rgb output");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const DevCamera dc = make_devcam(c, false);
    cudaEvent_t* ev = nullptr;
    if (flags & FGS_RENDER_STAGE_EVENTS) {
        if (!c->ev_ready) {
            for (int i = 0; i < kEventSlots; ++i)
                for (int k = 0; k <= kStages; ++k) FGS_CUDA(c, cudaEventCreate(&c->ev[i][k]));
            c->ev_ready = true;
        }
        ev = c->ev[c->ev_count % kEventSlots];
        ++c->ev_count;
    }
    const bool count = (flags & FGS_RENDER_COUNT) != 0;
    const bool pipelined = !out_is_device && (flags & FGS_RENDER_ASYNC);
    const size_t hw = (size_t)dc.width * dc.height;
    int slot = 0;
    if (pipelined) {
        if (flags & (FGS_RENDER_STATS | FGS_RENDER_COUNT))
            return fail(c, FGS_ERR_ARG, "FGS_RENDER_ASYNC does not combine with STATS or COUNT");
        if ((r = ensure_ring(c, hw))) return r;
        slot = c->ring_next;
    }
    int launches = enqueue_front(c, dc, s, ev, count);
    float* const img = pipelined ? c->ring[slot] : c->img;
    float* rgb_dst = out_is_device ? rgb_out : img;
    float* T_dst = out_is_device ? T_out : (T_out ? img + 3 * hw : nullptr);
    const bool keep = (flags & FGS_RENDER_KEEP) && !count;
    if (count) flags |= FGS_RENDER_STATS;
    // the image two frames back must have reached the host before it is overwritten
    if (pipelined && c->ring_busy[slot]) FGS_CUDA(c, cudaStreamWaitEvent(s, c->ev_copied[slot], 0));
    launch_blend(dc, c->ranges, c->vals1, c->splat, rgb_dst, T_dst, keep ? c->keep : nullptr, c->st, count, s);
    ++launches;
    if (ev) cudaEventRecord(ev[kStages], s);
    FGS_CUDA(c, cudaGetLastError());
    c->have_frame = true;
    c->frame_rendered = true;
    c->frame_kept = keep;
    if (pipelined) {
        // the copy runs on copy_stream while the caller's stream renders the next frame
        FGS_CUDA(c, cudaEventRecord(c->ev_blend[slot], s));
        FGS_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_blend[slot], 0));
        FGS_CUDA(c, cudaMemcpyAsync(rgb_out, img, 3 * hw * 4, cudaMemcpyDeviceToHost, c->copy_stream));
        if (T_out)
            FGS_CUDA(c, cudaMemcpyAsync(T_out, img + 3 * hw, hw * 4, cudaMemcpyDeviceToHost, c->copy_stream));
        FGS_CUDA(c, cudaEventRecord(c->ev_copied[slot], c->copy_stream));
        c->ring_busy[slot] = true;
        c->ring_next = slot ^ 1;
        if (st) {
            std::memset(st, 0, sizeof *st);
            st->n_launches = (uint32_t)launches;
        }
        return FGS_OK;
    }
    if (!out_is_device) {
        FGS_CUDA(c, cudaMemcpyAsync(rgb_out, c->img, 3 * hw * 4, cudaMemcpyDeviceToHost, s));
        if (T_out) FGS_CUDA(c, cudaMemcpyAsync(T_out, c->img + 3 * hw, hw * 4, cudaMemcpyDeviceToHost, s));
    }
    if (st) {
        std::memset(st, 0, sizeof *st);
        st->n_launches = (uint32_t)launches;
    }
    if ((flags & FGS_RENDER_STATS) || !out_is_device) {
        if ((r = read_state(c, s))) return r;
        if (st) {
            st->n_selected = c->st_host->M;
            st->n_pairs = c->st_host->n_pairs;
            st->device_status = c->st_host->status;
            st->blend_entries = c->st_host->blend_entries;
            st->blend_evals = c->st_host->blend_evals;
            st->blend_hits = c->st_host->blend_hits;
            st->blend_active = c->st_host->blend_active;
            st->n_emitting = c->st_host->n_emitting;
            st->filter_in_frustum = c->st_host->filter_in_frustum;
            st->filter_cov_nodes = c->st_host->filter_cov_nodes;
            st->filter_chunks_read = c->st_host->filter_chunks;
        }
        if ((r = latched_status(c))) {
            clear_status(c, s);
            return r;
        }
    }
    return FGS_OK;
}

int fgs_stage_times(fgs_ctx* c, int slot, float* ms_out)
{
    if (!c || !ms_out || slot < 0 || slot >= kEventSlots) return FGS_ERR_ARG;
    if (!c->ev_ready || (uint64_t)slot >= c->ev_count)
        return fail(c, FGS_ERR_ARG, "slot %d was never recorded", slot);
    DeviceGuard g(c->device);
    FGS_CUDA(c, cudaEventSynchronize(c->ev[slot][kStages]));
    for (int k = 0; k < kStages; ++k)
        FGS_CUDA(c, cudaEventElapsedTime(ms_out + k, c->ev[slot][k], c->ev[slot][k + 1]));
    return FGS_OK;
}

int fgs_stage_count(const fgs_ctx* c, uint64_t* count_out)
{
    if (!c || !count_out) return FGS_ERR_ARG;
    *count_out = c->ev_count;
    return FGS_OK;
}

int fgs_get_pairs(fgs_ctx* c, void* stream, uint64_t* keys_out, uint32_t* vals_out, uint64_t cap,
                  uint64_t* n_out, int out_is_device)
{
    if (!c || !n_out) return FGS_ERR_ARG;
    if (!c->have_frame) return fail(c, FGS_ERR_STATE, "no frame rendered");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r;
    if ((r = read_state(c, s))) return r;
    const uint64_t np = c->st_host->n_pairs;
    *n_out = np;
    const uint64_t n = std::min<uint64_t>(std::min<uint64_t>(np, c->pair_cap), cap);
    const unsigned long long* k = c->keys1;
    const uint32_t* v = c->vals1;
    const cudaMemcpyKind kind = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (n && keys_out) FGS_CUDA(c, cudaMemcpyAsync(keys_out, k, n * 8, kind, s));
    if (n && vals_out) FGS_CUDA(c, cudaMemcpyAsync(vals_out, v, n * 4, kind, s));
    FGS_CUDA(c, cudaStreamSynchronize(s));
    if ((r = latched_status(c))) return r;
    if (np > cap) return fail(c, FGS_ERR_CAPACITY, "N_P %llu exceeds cap %llu", (unsigned long long)np,
                              (unsigned long long)cap);
    return FGS_OK;
}

int fgs_get_splats(fgs_ctx* c, void* stream, float* out, uint32_t cap, uint32_t* M_out,
                   int out_is_device)
{
    if (!c || !M_out) return FGS_ERR_ARG;
    if (!c->have_frame) return fail(c, FGS_ERR_STATE, "no frame rendered");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r;
    if ((r = read_state(c, s))) return r;
    const uint32_t M = c->st_host->M;
    *M_out = M;
    const uint64_t n = std::min<uint64_t>(M, cap);
    if (n && out)
        FGS_CUDA(c, cudaMemcpyAsync(out, c->splat, n * kSplatStride * 4,
                                    out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    FGS_CUDA(c, cudaStreamSynchronize(s));
    if (M > cap) return fail(c, FGS_ERR_CAPACITY, "M %u exceeds cap %u", M, cap);
    return FGS_OK;
}

namespace {

// The current camera through the KPC blend (Eq. 5-7); force_3sigma selects the
// calibration footprint, otherwise the context's shrink mode applies.
int kpc_view(fgs_ctx* c, void* stream, bool force_3sigma, double* gbar_out, float* kpc_out,
             uint64_t kpc_cap, float* G_out, int out_is_device)
{
    int r = check_ready(c);
    if (r) return r;
    if (!gbar_out) return fail(c, FGS_ERR_ARG, "null gbar output");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const DevCamera dc = make_devcam(c, force_3sigma);
    enqueue_front(c, dc, s, nullptr);
    FGS_CUDA(c, cudaMemsetAsync(c->kpc, 0, c->pair_cap * 4, s));
    launch_blend_kpc(dc, c->ranges, c->vals1, c->splat, c->kpc, c->G, c->st, s);
    FGS_CUDA(c, cudaGetLastError());
    c->have_frame = true;
    c->frame_rendered = false;
    c->frame_kept = false;
    if ((r = read_state(c, s))) return r;
    if ((r = latched_status(c))) {
        clear_status(c, s);
        return r;
    }
    const FrameState& h = *c->st_host;
    const size_t tiles = (size_t)dc.tiles_x * dc.tiles_y;
    std::vector<float> Gh(tiles);
    FGS_CUDA(c, cudaMemcpyAsync(Gh.data(), c->G, tiles * 4, cudaMemcpyDeviceToHost, s));
    const cudaMemcpyKind kind = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const uint64_t np = std::min<uint64_t>(h.n_pairs, c->pair_cap);
    if (kpc_out && np) FGS_CUDA(c, cudaMemcpyAsync(kpc_out, c->kpc, std::min(np, kpc_cap) * 4, kind, s));
    if (G_out) FGS_CUDA(c, cudaMemcpyAsync(G_out, c->G, tiles * 4, kind, s));
    FGS_CUDA(c, cudaStreamSynchronize(s));
    // Eq. 7: mean of G over the tiles that have pairs (tile order, float64)
    double sum = 0.0;
    size_t used = 0;
    for (size_t i = 0; i < tiles; ++i)
        if (!std::isnan(Gh[i])) {
            sum += (double)Gh[i];
            ++used;
        }
    *gbar_out = used ? sum / (double)used : NAN;
    return FGS_OK;
}

}  // namespace

int fgs_calibrate_view(fgs_ctx* c, void* stream, double* gbar_out, float* kpc_out, uint64_t kpc_cap,
                       float* G_out, int out_is_device)
{
    // calibration uses the 3-sigma footprint
    return kpc_view(c, stream, true, gbar_out, kpc_out, kpc_cap, G_out, out_is_device);
}

int fgs_kpc_view(fgs_ctx* c, void* stream, double* gbar_out, float* kpc_out, uint64_t kpc_cap,
                 float* G_out, int out_is_device)
{
    return kpc_view(c, stream, false, gbar_out, kpc_out, kpc_cap, G_out, out_is_device);
}

int fgs_calibrate_gtc(fgs_ctx* c, void* stream, const fgs_camera* views, int n_views, float lambda_G,
                      double* gbar_views_out, float* tau_out, float* ln_tau_out)
{
    if (!c || !views || n_views < 1 || !tau_out || !ln_tau_out) return FGS_ERR_ARG;
    if (!(lambda_G > 0) || !std::isfinite(lambda_G)) return fail(c, FGS_ERR_ARG, "lambda_G invalid");
    double sum = 0.0;
    int used = 0;
    for (int v = 0; v < n_views; ++v) {
        int r = fgs_set_camera(c, views + v);
        if (r) return r;
        double gbar = NAN;
        r = fgs_calibrate_view(c, stream, &gbar, nullptr, 0, nullptr, 0);
        if (r) return r;
        if (gbar_views_out) gbar_views_out[v] = gbar;
        if (std::isfinite(gbar)) {   // a view without any pair has no G_v
            sum += gbar;
            ++used;
        }
    }
    if (used == 0) return fail(c, FGS_ERR_ARG, "no calibration view produced pairs");
    const double G = sum / used;                                   // Eq. 8
    *tau_out = (float)((double)lambda_G / G);
    *ln_tau_out = (float)(std::log((double)lambda_G) - std::log(G));
    return FGS_OK;
}

int fgs_eval_exp(const float* x, float* y, uint64_t n, void* stream)
{
    if ((!x || !y) && n) return FGS_ERR_ARG;
    if (n == 0) return FGS_OK;
    launch_eval_exp(x, y, n, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}

int fgs_probe_wait_timeout(fgs_ctx* c, void* stream, uint32_t* site_out)
{
    if (!c) return FGS_ERR_ARG;
    if (!c->has_tree) return fail(c, FGS_ERR_STATE, "no tree loaded");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r;
    if ((r = clear_status(c, s))) return r;
    launch_wait_probe(c->lb_compact, c->st, s);
    FGS_CUDA(c, cudaGetLastError());
    if ((r = read_state(c, s))) return r;
    if (site_out) *site_out = c->st_host->status_info;
    r = latched_status(c);
    if (r) clear_status(c, s);
    FGS_CUDA(c, cudaStreamSynchronize(s));
    return r;
}

// ---------------------------------------------------------------------------
// differentiable form
// ---------------------------------------------------------------------------
namespace {

bool is_device_ptr(const void* p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

int check_param_ptrs(fgs_ctx* c, const void* const* ptrs, const char* const* names, int n)
{
    for (int i = 0; i < n; ++i)
        if (!is_device_ptr(ptrs[i], c->device))
            return fail(c, FGS_ERR_ARG, "%s is not a device pointer on device %d", names[i], c->device);
    return FGS_OK;
}

}  // namespace

int fgs_update_params(fgs_ctx* c, void* stream, const fgs_gauss_params* p)
{
    if (!c || !p) return FGS_ERR_ARG;
    if (!c->has_tree) return fail(c, FGS_ERR_STATE, "no tree loaded");
    DeviceGuard g(c->device);
    const void* ptrs[] = {p->mu, p->log_scale, p->quat, p->logit, p->sh};
    const char* names[] = {"mu", "log_scale", "quat", "logit", "sh"};
    int r = check_param_ptrs(c, ptrs, names, 5);
    if (r) return r;
    c->have_frame = false;
    const int blocks = (int)std::min<uint64_t>((c->tree.n + 255) / 256, (uint64_t)c->sms * 8);
    launch_prep_params(c->tree, p->mu, p->log_scale, p->quat, p->logit, p->sh, std::max(blocks, 1),
                       (cudaStream_t)stream);
    launch_chunk_boxes(c->tree, c->sms, (cudaStream_t)stream);     // the centres changed
    FGS_CUDA(c, cudaGetLastError());
    return FGS_OK;
}

int fgs_backward(fgs_ctx* c, void* stream, const float* dL_drgb, const fgs_gauss_params* p,
                 const fgs_gauss_grads* gr, uint32_t flags)
{
    int r = check_ready(c);
    if (r) return r;
    if (!p || !gr) return fail(c, FGS_ERR_ARG, "null parameter or gradient struct");
    if (!c->have_frame || !c->frame_rendered) return fail(c, FGS_ERR_STATE, "no rendered frame to differentiate");
    DeviceGuard g(c->device);
    const void* ptrs[] = {dL_drgb, p->mu, p->log_scale, p->quat, p->logit, p->sh,
                          gr->mu, gr->log_scale, gr->quat, gr->logit, gr->sh};
    const char* names[] = {"dL_drgb", "mu", "log_scale", "quat", "logit", "sh",
                           "grad mu", "grad log_scale", "grad quat", "grad logit", "grad sh"};
    if ((r = check_param_ptrs(c, ptrs, names, 11))) return r;
    if (c->gsplat_rows < c->tree.n) {
        if ((r = grow(c, (void**)&c->gsplat, (size_t)c->tree.n * 12 * sizeof(float)))) return r;
        c->gsplat_rows = c->tree.n;
    }
    const DevCamera dc = make_devcam(c, false);
    cudaStream_t s = (cudaStream_t)stream;
    const float* params[5] = {p->mu, p->log_scale, p->quat, p->logit, p->sh};
    float* grads[5] = {gr->mu, gr->log_scale, gr->quat, gr->logit, gr->sh};
    launch_backward(c->tree, dc, c->ranges, c->vals1, c->splat, c->keep, c->frame_kept, c->sel,
                    dL_drgb, c->gsplat, params, grads, (flags & FGS_BACKWARD_ACCUMULATE) != 0, c->sms, c->st,
                    s);
    FGS_CUDA(c, cudaGetLastError());
    return FGS_OK;
}

// ---------------------------------------------------------------------------
// batched multi-view form
// ---------------------------------------------------------------------------
int fgs_batch_setup(fgs_ctx* c, const fgs_camera* views, int n_views, const int32_t* tile_shapes,
                    uint64_t sel_capacity, uint64_t pair_capacity)
{
    if (!c || !views || n_views < 1 || n_views > 64) return FGS_ERR_ARG;
    if (!c->has_tree) return fail(c, FGS_ERR_STATE, "no tree loaded");
    for (int v = 0; v < n_views; ++v)
        if (!valid_camera(views + v)) return fail(c, FGS_ERR_ARG, "view %d: invalid camera", v);
    if ((uint64_t)n_views * c->tree.n_pad >= (1ull << 32))
        return fail(c, FGS_ERR_ARG, "views x nodes exceeds 2^32 selection entries");
    DeviceGuard g(c->device);
    auto& b = c->batch;
    if (b.graph) {
        cudaGraphExecDestroy(b.graph);
        b.graph = nullptr;
    }
    b.V = n_views;
    b.have_frame = false;
    b.cams.assign(views, views + n_views);
    b.tile_w.assign(n_views, c->params.tile_w);
    b.tile_h.assign(n_views, c->params.tile_h);
    b.warp_w.assign(n_views, c->params.blend_warp_w);
    if (tile_shapes) {
        for (int v = 0; v < n_views; ++v) {
            const int tw = tile_shapes[3 * v], th = tile_shapes[3 * v + 1];
            const int ww = tile_shapes[3 * v + 2] ? tile_shapes[3 * v + 2] : 8;
            if (!is_pow2(tw) || !is_pow2(th) || tw * th != 256 || tw < 8 || th < 4 ||
                (ww != 8 && ww != 4) || th < 32 / ww)
                return fail(c, FGS_ERR_ARG, "view %d: tile %dx%d / warp %d not supported", v, tw, th, ww);
            b.tile_w[v] = tw;
            b.tile_h[v] = th;
            b.warp_w[v] = ww;
        }
    }
    b.tile_base.assign(n_views + 1, 0);
    b.img_off.assign(n_views + 1, 0);
    for (int v = 0; v < n_views; ++v) {
        const uint32_t tx = (views[v].width + b.tile_w[v] - 1) / b.tile_w[v];
        const uint32_t ty = (views[v].height + b.tile_h[v] - 1) / b.tile_h[v];
        b.tile_base[v + 1] = b.tile_base[v] + tx * ty;
        b.img_off[v + 1] = b.img_off[v] + (unsigned long long)views[v].width * views[v].height;
    }
    b.total_tiles = b.tile_base[n_views];
    const uint64_t sel_cap = sel_capacity ? sel_capacity : std::min<uint64_t>((uint64_t)n_views * c->tree.n_pad, 64ull << 20);
    const uint64_t pair_cap = pair_capacity ? pair_capacity : (128ull << 20);
    if (pair_cap > kMaxPairCap) return fail(c, FGS_ERR_ARG, "pair capacity too large");
    const size_t n_words = c->tree.n_pad / 32;
    int r;
    if ((r = grow(c, (void**)&b.d_cams, sizeof(DevCamera) * n_views))) return r;
    if (!b.h_cams) FGS_CUDA(c, cudaMallocHost((void**)&b.h_cams, sizeof(DevCamera) * 64));
    if ((r = grow(c, (void**)&b.d_tile_base, 4 * (n_views + 1)))) return r;
    if ((r = grow(c, (void**)&b.d_img_off, 8 * (n_views + 1)))) return r;
    if ((r = grow(c, (void**)&b.pbits, 4 * n_words * n_views))) return r;
    if ((r = grow(c, (void**)&b.selbits, 4 * n_words * n_views))) return r;
    if ((r = grow(c, (void**)&b.lb_compact, 8 * (n_words * n_views / kCompactWords + 2)))) return r;
    if ((r = grow(c, (void**)&b.lb_scan, 8 * tile_scan_lookback_entries(b.total_tiles)))) return r;
    if (sel_cap != b.sel_cap) {
        if ((r = grow(c, (void**)&b.sel, 4 * sel_cap))) return r;
        if ((r = grow(c, (void**)&b.splat, 4 * kSplatStride * sel_cap))) return r;
        if ((r = grow(c, (void**)&b.foot, sizeof(uint4) * sel_cap))) return r;
        b.sel_cap = sel_cap;
    }
    if (pair_cap != b.pair_cap) {
        const size_t n = pair_cap + 8;
        if ((r = grow(c, (void**)&b.items, 8 * n))) return r;
        if ((r = grow(c, (void**)&b.keys, 8 * n))) return r;
        if ((r = grow(c, (void**)&b.vals, 4 * n))) return r;
        b.pair_cap = pair_cap;
    }
    if ((r = grow(c, (void**)&b.ranges, sizeof(uint2) * b.total_tiles))) return r;
    if ((r = grow(c, (void**)&b.tile_cnt, 4 * b.total_tiles))) return r;
    if ((r = grow(c, (void**)&b.large, 4 * b.total_tiles))) return r;
    if (!b.st) {
        if ((r = grow(c, (void**)&b.st, sizeof(FrameState)))) return r;
    }
    FGS_CUDA(c, cudaMemcpy(b.d_tile_base, b.tile_base.data(), 4 * (n_views + 1), cudaMemcpyHostToDevice));
    FGS_CUDA(c, cudaMemcpy(b.d_img_off, b.img_off.data(), 8 * (n_views + 1), cudaMemcpyHostToDevice));
    return FGS_OK;
}

int fgs_batch_set_cameras(fgs_ctx* c, const fgs_camera* views, int n_views)
{
    if (!c || !views) return FGS_ERR_ARG;
    auto& b = c->batch;
    if (b.V == 0) return fail(c, FGS_ERR_STATE, "no batch set up");
    if (n_views != b.V) return fail(c, FGS_ERR_ARG, "batch has %d views", b.V);
    for (int v = 0; v < n_views; ++v) {
        if (!valid_camera(views + v)) return fail(c, FGS_ERR_ARG, "view %d: invalid camera", v);
        if (views[v].width != b.cams[v].width || views[v].height != b.cams[v].height)
            return fail(c, FGS_ERR_ARG, "view %d: resolution differs from the batch set-up", v);
    }
    b.cams.assign(views, views + n_views);
    return FGS_OK;
}

int fgs_batch_image_offsets(const fgs_ctx* c, uint64_t* offsets_out)
{
    if (!c || !offsets_out) return FGS_ERR_ARG;
    const auto& b = c->batch;
    if (b.V == 0) return FGS_ERR_STATE;
    for (int v = 0; v <= b.V; ++v) offsets_out[v] = b.img_off[v];
    return FGS_OK;
}

namespace {

void enqueue_batch(fgs_ctx* c, float* rgb, float* T, cudaStream_t s)
{
    auto& b = c->batch;
    launch_batch_front(c->tree, b.d_cams, b.V, b.total_tiles, b.d_tile_base, b.pbits, b.selbits, b.sel,
                       (uint32_t)b.sel_cap, b.splat, b.foot, b.tile_cnt, b.large, b.items, b.keys, b.vals,
                       b.pair_cap, b.lb_compact, b.lb_scan, b.ranges, b.st, c->sms, s);
    launch_batch_blend(b.d_cams, b.V, b.total_tiles, b.d_tile_base, b.d_img_off, b.ranges, b.vals, b.splat,
                       rgb, T, b.st, s);
}

}  // namespace

int fgs_render_batch(fgs_ctx* c, void* stream, float* rgb_out, float* T_out, uint32_t flags,
                     fgs_stats* st)
{
    if (!c || !rgb_out) return FGS_ERR_ARG;
    auto& b = c->batch;
    if (b.V == 0) return fail(c, FGS_ERR_STATE, "no batch set up");
    if (!c->has_tree) return fail(c, FGS_ERR_STATE, "no tree loaded");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    for (int v = 0; v < b.V; ++v) {
        DevCamera d = make_devcam_for(c, b.cams[v], b.tile_w[v], b.tile_h[v], b.warp_w[v]);
        b.h_cams[v] = d;
    }
    FGS_CUDA(c, cudaMemcpyAsync(b.d_cams, b.h_cams, sizeof(DevCamera) * b.V, cudaMemcpyHostToDevice, s));
    const int launches = 9;
    if (flags & FGS_BATCH_GRAPH) {
        if (!b.graph || b.graph_rgb != rgb_out || b.graph_T != T_out) {
            if (b.graph) {
                cudaGraphExecDestroy(b.graph);
                b.graph = nullptr;
            }
            cudaStream_t cs;
            FGS_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            FGS_CUDA(c, cudaStreamSynchronize(s));
            cudaGraph_t graph = nullptr;
            FGS_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            enqueue_batch(c, rgb_out, T_out, cs);
            const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            if (ce != cudaSuccess)
                return fail(c, FGS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&b.graph, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess)
                return fail(c, FGS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
            b.graph_rgb = rgb_out;
            b.graph_T = T_out;
        }
        FGS_CUDA(c, cudaGraphLaunch(b.graph, s));
    } else {
        enqueue_batch(c, rgb_out, T_out, s);
    }
    FGS_CUDA(c, cudaGetLastError());
    b.have_frame = true;
    if (st) {
        std::memset(st, 0, sizeof *st);
        st->n_launches = (uint32_t)launches;
    }
    if (flags & FGS_RENDER_STATS) {
        FGS_CUDA(c, cudaMemcpyAsync(c->st_host, b.st, sizeof(FrameState), cudaMemcpyDeviceToHost, s));
        FGS_CUDA(c, cudaStreamSynchronize(s));
        if (st) {
            st->n_selected = c->st_host->M;
            st->n_pairs = c->st_host->n_pairs;
            st->device_status = c->st_host->status;
        }
        if (c->st_host->status) {
            const int code = c->st_host->status == kErrCapacity ? FGS_ERR_CAPACITY : FGS_ERR_TIMEOUT;
            FGS_CUDA(c, cudaMemsetAsync(&b.st->status, 0, 8, s));
            return fail(c, code, "batch: device status %d (N_P %llu, selected %u)", c->st_host->status,
                        (unsigned long long)c->st_host->n_pairs, c->st_host->M);
        }
        if (c->st_host->M > b.sel_cap)
            return fail(c, FGS_ERR_CAPACITY, "batch selection %u exceeds capacity %llu", c->st_host->M,
                        (unsigned long long)b.sel_cap);
    }
    return FGS_OK;
}

int fgs_batch_get_frame(fgs_ctx* c, void* stream, uint32_t* entries_out, float* splat_out,
                        uint64_t sel_cap, uint64_t* M_out, uint64_t* keys_out, uint32_t* vals_out,
                        uint64_t pair_cap, uint64_t* NP_out, uint32_t* node_stride_out,
                        uint32_t* tile_base_out)
{
    if (!c || !M_out || !NP_out) return FGS_ERR_ARG;
    auto& b = c->batch;
    if (b.V == 0 || !b.have_frame) return fail(c, FGS_ERR_STATE, "no batch rendered");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    FGS_CUDA(c, cudaMemcpyAsync(c->st_host, b.st, sizeof(FrameState), cudaMemcpyDeviceToHost, s));
    FGS_CUDA(c, cudaStreamSynchronize(s));
    const uint64_t M = c->st_host->M, np = c->st_host->n_pairs;
    *M_out = M;
    *NP_out = np;
    if (node_stride_out) *node_stride_out = (uint32_t)c->tree.n_pad;
    if (tile_base_out)
        for (int v = 0; v <= b.V; ++v) tile_base_out[v] = b.tile_base[v];
    const uint64_t m = std::min<uint64_t>(std::min<uint64_t>(M, b.sel_cap), sel_cap);
    const uint64_t n = std::min<uint64_t>(std::min<uint64_t>(np, b.pair_cap), pair_cap);
    if (m && entries_out) FGS_CUDA(c, cudaMemcpyAsync(entries_out, b.sel, m * 4, cudaMemcpyDeviceToHost, s));
    if (m && splat_out)
        FGS_CUDA(c, cudaMemcpyAsync(splat_out, b.splat, m * kSplatStride * 4, cudaMemcpyDeviceToHost, s));
    if (n && keys_out)
        FGS_CUDA(c, cudaMemcpyAsync(keys_out, b.keys, n * 8, cudaMemcpyDeviceToHost, s));
    if (n && vals_out)
        FGS_CUDA(c, cudaMemcpyAsync(vals_out, b.vals, n * 4, cudaMemcpyDeviceToHost, s));
    FGS_CUDA(c, cudaStreamSynchronize(s));
    if (c->st_host->status)
        return fail(c, c->st_host->status == kErrCapacity ? FGS_ERR_CAPACITY : FGS_ERR_TIMEOUT,
                    "batch: device status %d", c->st_host->status);
    if (((entries_out || splat_out) && M > sel_cap) || ((keys_out || vals_out) && np > pair_cap))
        return fail(c, FGS_ERR_CAPACITY, "batch M %llu / N_P %llu exceed caps %llu / %llu",
                    (unsigned long long)M, (unsigned long long)np, (unsigned long long)sel_cap,
                    (unsigned long long)pair_cap);
    return FGS_OK;
}

int fgs_sync(fgs_ctx* c, void* stream)
{
    if (!c) return FGS_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r;
    if ((r = read_state(c, s))) return r;
    r = latched_status(c);
    if (r) clear_status(c, s);
    FGS_CUDA(c, cudaStreamSynchronize(s));
    if (c->copy_stream) FGS_CUDA(c, cudaStreamSynchronize(c->copy_stream));   // pipelined host copies
    return r;
}

}  // extern "C"
