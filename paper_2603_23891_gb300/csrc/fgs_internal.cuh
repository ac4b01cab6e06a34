// Internal declarations of the FilterGS CUDA library (sm_103a).
//
// Decision-exact arithmetic: every value that decides an integer result
// (frustum test, R&L predicate, tile rectangle, depth key, shrink radius,
// blend skip/stop) is computed with explicitly rounded binary32 intrinsics
// (__fmul_rn, __fadd_rn, ... never contracted into FMA) in one fixed order,
// so that selections, keys and pair lists are reproducible bit for bit on any
// IEEE machine that follows the same order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace fgs {

constexpr int kStages = 7;
constexpr uint32_t kApPad = 0xFFFFFFFFu;
constexpr int kSplatStride = 12;          // floats per splat record (48 B)
constexpr int kSegSmall = 256;            // pairs of a tile sorted by one warp in registers
constexpr int kSegSmem = 2048;            // pairs of a tile sorted by one block in shared memory
constexpr int kFilterTile = 4096;         // node arrays are padded to a multiple of this
constexpr int kCompactWords = 1024;       // 32-bit selection words per compaction tile (32K nodes)
constexpr int kSelTileWords = 256;        // words per counted tile (the Ancestor filter's sel_cnt)
constexpr int kAncCacheWords = 4096;      // P-bit words of the lowest node ids kept in shared memory
constexpr int kProjThreads = 256;         // selected Gaussians per projection tile
constexpr uint64_t kSpinLimit = 1ull << 24;   // bounded spin-waits

// device status codes (mirrors FGS_ERR_* of the C ABI)
constexpr int kErrCapacity = -4;
constexpr int kErrTimeout = -5;

struct DevCamera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float tan_half_x, tan_half_y;
    float campos[3];
    int32_t width, height;
    // derived on the host (exact: products by powers of two, integer ceil)
    int32_t tiles_x, tiles_y;
    int32_t tile_w, tile_h;
    int32_t tile_shift_x, tile_shift_y;
    float tau_R;
    int32_t shrink;
    float tau, ln_tau;
    float bg[3];
    int32_t warp_shift;        // blend warps cover (1 << warp_shift) x (32 >> warp_shift) pixels
};

// Tree on the device (SoA; arrays padded to a multiple of 128 nodes).
struct DevTree {
    uint32_t n;
    uint32_t n_pad;
    uint32_t depth;
    uint32_t sh_degree;
    uint32_t sh_stride;        // floats per node in sh (K*3 rounded up to 4)
    const float* mu;           // [3][n_pad]
    const float* cov;          // [6][n_pad]
    const float* opacity;      // [n_pad]
    const float* ln_opacity;   // [n_pad]
    const float* sh;           // [n_pad][sh_stride]
    const uint32_t* leaf_bits; // [n_pad/32]
    const uint32_t* ap;        // [depth][n_pad]
    // the projection's gather copy, node-major: {mu.x, mu.y, mu.z, alpha0},
    // {xx, xy, xz, yy}, {yz, zz, ln alpha0, 0}
    const float4* attr;        // [n_pad][3]
    // per 128 consecutive nodes (one warp's chunk in the R&L filter): the box of
    // their centres, {lo.x, lo.y, lo.z, 0}, {hi.x, hi.y, hi.z, 0}; lo.x > hi.x for a
    // chunk of padding only
    const float4* cbox;        // [n_pad / 128][2]
};

// Per-frame device state (one per context).
struct FrameState {
    uint32_t epoch;            // bumped once per frame; tags look-back entries
    uint32_t M;                // selected nodes
    unsigned long long n_pairs;  // emitted pairs (true count, may exceed capacity)
    uint32_t tickets[16];      // dynamic tile counters (one per kernel use)
    int32_t status;            // latched error (0 = ok)
    uint32_t status_info;
    uint32_t reserved0;
    unsigned long long blend_entries;     // lockstep warp steps of the list walk (counting frames only)
    unsigned long long blend_evals;       // pixel-Gaussian evaluations (lanes not yet stopped)
    unsigned long long blend_hits;        // evaluations that reached the alpha / T update
    unsigned long long blend_active;      // lockstep steps where some lane reached it
    uint32_t n_emitting;                  // selected Gaussians with at least one pair
    unsigned long long filter_in_frustum; // counting frames: nodes in the frustum
    unsigned long long filter_cov_nodes;  // counting frames: in-frustum internal nodes
    unsigned long long filter_chunks;     // counting frames: 128-node chunks whose centres R&L read

};

// Ticket slots
enum : int { kTicketCompact = 0, kTicketSegSort = 2, kTicketScan = 4, kTicketLarge = 5 };

// ---------------------------------------------------------------------
// decision-exact binary32 helpers
// ---------------------------------------------------------------------
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }

__device__ __forceinline__ float ff(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// e^x in binary32 for x in [-87, 0]: Cody & Waite argument reduction
// (x = k ln2 + r, k the integer nearest x log2(e), taken from the binary32 sum
// x log2(e) + 1.5 * 2^23 formed with one rounding; ln 2 split into a short
// leading part and a correction), the degree-7 Taylor polynomial of e^r by
// Horner's rule with fused multiply-adds, scaled by 2^k from exponent bits
// (k = the low bits of that sum; k + 127 lies in [1, 254] for x >= -87).
// Explicitly rounded operations, so the bits do not depend on the compiler.
__device__ __forceinline__ float exp_hit(float x)
{
    const float t = ff(x, 1.44269504088896341f, 12582912.0f);
    const float kf = fs(t, 12582912.0f);
    float r = ff(kf, -0.693359375f, x);
    r = ff(kf, 2.12194440e-4f, r);
    float p = 1.98412698412698413e-4f;
    p = ff(p, r, 1.38888888888888889e-3f);
    p = ff(p, r, 8.33333333333333333e-3f);
    p = ff(p, r, 4.16666666666666667e-2f);
    p = ff(p, r, 1.66666666666666667e-1f);
    p = ff(p, r, 0.5f);
    p = ff(p, r, 1.0f);
    p = ff(p, r, 1.0f);
    const float two_k = __uint_as_float((__float_as_uint(t) + (uint32_t)(127 - 0x4B400000)) << 23);
    return fm(p, two_k);
}

// The same for x <= 0 or NaN (0 below -87); for x <= 0 the same as exp_cw below.
__device__ __forceinline__ float exp_nonpos(float x)
{
    const float y = exp_hit(x);
    return x < -87.0f ? 0.0f : y;
}

// e^x in binary32 for any x: 0 below -87, infinity above 88.
__device__ __forceinline__ float exp_cw(float x)
{
    if (x > 88.0f) return __int_as_float(0x7f800000);
    return exp_nonpos(x);
}

// Screen-space view of one node: camera-space centre, frustum test and the
// 2D covariance J W Sigma W^T J^T + 0.3 I (EWA), larger eigenvalue.
struct NodeView {
    bool in_frustum;
    float vx, vy, vz;
    float a, b, c;
    float lam;
};

__device__ __forceinline__ void camera_space(const DevCamera& cam, float mx, float my, float mz,
                                             float& vx, float& vy, float& vz)
{
    vx = fa(fa(fa(fm(cam.R[0], mx), fm(cam.R[1], my)), fm(cam.R[2], mz)), cam.t[0]);
    vy = fa(fa(fa(fm(cam.R[3], mx), fm(cam.R[4], my)), fm(cam.R[5], mz)), cam.t[1]);
    vz = fa(fa(fa(fm(cam.R[6], mx), fm(cam.R[7], my)), fm(cam.R[8], mz)), cam.t[2]);
}

// Frustum: depth above 0.2 and the centre within 1.3x the half-FOV tangents.
__device__ __forceinline__ bool frustum_test(const DevCamera& cam, float vx, float vy, float vz,
                                             float& txtz, float& tytz)
{
    if (!(vz > 0.2f)) return false;
    const float limx = fm(1.3f, cam.tan_half_x);
    const float limy = fm(1.3f, cam.tan_half_y);
    txtz = fd(vx, vz);
    tytz = fd(vy, vz);
    return txtz >= -limx && txtz <= limx && tytz >= -limy && tytz <= limy;
}

// Whether every centre in the box [lo, hi] fails the frustum test (§3.2's
// in-frustum condition: depth above 0.2, |x / z| and |y / z| within 1.3 times
// the half-FOV tangents), so that the R&L filter can skip reading the chunk: the
// box lies beyond one of the five planes x = L z, x = -L z, y = L z, y = -L z,
// z = 0.2 (a point beyond a side plane either has x / z beyond L or a depth
// below the near plane).  Exact for the per-node binary32 test: a plane counts
// only if the box clears it by a margin of 1e-3 times the magnitudes involved,
// a thousand times the rounding of the camera transform and the divisions.
struct FrustumPlanes {
    float4 p[5];      // n.x, n.y, n.z, d: outside where n . p + d > 0
    float scale;      // 1 + the larger guard-banded tangent
    float tt;         // |t|_1 of the camera translation
};

__device__ __forceinline__ void frustum_planes(const DevCamera& cam, FrustumPlanes& F)
{
    const float Lx = fm(1.3f, cam.tan_half_x), Ly = fm(1.3f, cam.tan_half_y);
    const float* R = cam.R;
    const float* t = cam.t;
    // right, left, bottom, top, near
    F.p[0] = make_float4(R[0] - Lx * R[6], R[1] - Lx * R[7], R[2] - Lx * R[8], t[0] - Lx * t[2]);
    F.p[1] = make_float4(-R[0] - Lx * R[6], -R[1] - Lx * R[7], -R[2] - Lx * R[8], -t[0] - Lx * t[2]);
    F.p[2] = make_float4(R[3] - Ly * R[6], R[4] - Ly * R[7], R[5] - Ly * R[8], t[1] - Ly * t[2]);
    F.p[3] = make_float4(-R[3] - Ly * R[6], -R[4] - Ly * R[7], -R[5] - Ly * R[8], -t[1] - Ly * t[2]);
    F.p[4] = make_float4(-R[6], -R[7], -R[8], 0.2f - t[2]);
    F.scale = 1.0f + fmaxf(Lx, Ly);
    F.tt = fabsf(t[0]) + fabsf(t[1]) + fabsf(t[2]);
}

__device__ __forceinline__ bool chunk_outside(const FrustumPlanes& F, float4 lo, float4 hi)
{
    if (lo.x > hi.x) return true;                          // padding only
    const float ax = fmaxf(fabsf(lo.x), fabsf(hi.x)), ay = fmaxf(fabsf(lo.y), fabsf(hi.y));
    const float az = fmaxf(fabsf(lo.z), fabsf(hi.z));
    const float margin = 1e-3f * ((ax + ay + az + F.tt) * F.scale + 1.0f);
    bool out = false;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float4 q = F.p[k];
        const float m = q.w + fminf(q.x * lo.x, q.x * hi.x) + fminf(q.y * lo.y, q.y * hi.y) +
                        fminf(q.z * lo.z, q.z * hi.z);
        out |= m > margin;
    }
    return out;
}

// Sigma_2D and lambda_max for an in-frustum node.  s = {xx, xy, xz, yy, yz, zz}.
__device__ __forceinline__ void ewa_cov2d(const DevCamera& cam, float vz, float txtz, float tytz,
                                          const float s[6], float& a, float& b, float& c, float& lam)
{
    const float limx = fm(1.3f, cam.tan_half_x);
    const float limy = fm(1.3f, cam.tan_half_y);
    const float clx = fminf(limx, fmaxf(-limx, txtz));
    const float cly = fminf(limy, fmaxf(-limy, tytz));
    const float txc = fm(clx, vz);
    const float tyc = fm(cly, vz);
    const float tz2 = fm(vz, vz);
    const float j00 = fd(cam.fx, vz);
    const float j11 = fd(cam.fy, vz);
    const float j02 = -fd(fm(cam.fx, txc), tz2);
    const float j12 = -fd(fm(cam.fy, tyc), tz2);
    const float* R = cam.R;
    const float m00 = fa(fm(j00, R[0]), fm(j02, R[6]));
    const float m01 = fa(fm(j00, R[1]), fm(j02, R[7]));
    const float m02 = fa(fm(j00, R[2]), fm(j02, R[8]));
    const float m10 = fa(fm(j11, R[3]), fm(j12, R[6]));
    const float m11 = fa(fm(j11, R[4]), fm(j12, R[7]));
    const float m12 = fa(fm(j11, R[5]), fm(j12, R[8]));
    const float s00 = s[0], s01 = s[1], s02 = s[2], s11 = s[3], s12 = s[4], s22 = s[5];
    const float u0 = fa(fa(fm(s00, m00), fm(s01, m01)), fm(s02, m02));
    const float u1 = fa(fa(fm(s01, m00), fm(s11, m01)), fm(s12, m02));
    const float u2 = fa(fa(fm(s02, m00), fm(s12, m01)), fm(s22, m02));
    const float w0 = fa(fa(fm(s00, m10), fm(s01, m11)), fm(s02, m12));
    const float w1 = fa(fa(fm(s01, m10), fm(s11, m11)), fm(s12, m12));
    const float w2 = fa(fa(fm(s02, m10), fm(s12, m11)), fm(s22, m12));
    a = fa(fa(fa(fm(m00, u0), fm(m01, u1)), fm(m02, u2)), 0.3f);
    b = fa(fa(fm(m10, u0), fm(m11, u1)), fm(m12, u2));
    c = fa(fa(fa(fm(m10, w0), fm(m11, w1)), fm(m12, w2)), 0.3f);
    const float det = fs(fm(a, c), fm(b, b));
    const float mid = fm(0.5f, fa(a, c));
    float disc = fs(fm(mid, mid), det);
    disc = disc > 0.1f ? disc : 0.1f;
    lam = fa(mid, fsq(disc));
}

// ---------------------------------------------------------------------
// bounded look-back / spin helpers
// ---------------------------------------------------------------------
// Look-back entries carry their whole payload (epoch tag, flag, count) in one
// 64-bit word and publish no other data, so relaxed device-scope accesses
// suffice (no acquire / release ordering is needed around them).
__device__ __forceinline__ unsigned long long ld_lb_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_lb_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// look-back entry: [63:34] epoch (30 bits) | [33:32] flag | [31:0] value
constexpr unsigned long long kFlagAgg = 1ull;
constexpr unsigned long long kFlagIncl = 2ull;
__device__ __forceinline__ unsigned long long lb_pack(uint32_t epoch, unsigned long long flag, uint32_t v)
{
    return ((unsigned long long)(epoch & 0x3FFFFFFFu) << 34) | (flag << 32) | v;
}

// Programmatic dependent launch: the frame's kernels are launched with
// programmatic stream serialisation, so a kernel's blocks may start while its
// predecessor drains.  Every kernel calls grid_dep_wait() before it touches
// anything a predecessor wrote (it returns once the predecessor grid has
// completed and its writes are visible), and grid_dep_trigger() once it no
// longer needs to hold the next kernel back.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void set_status(FrameState* st, int code, uint32_t info)
{
    if (atomicCAS(&st->status, 0, code) == 0) st->status_info = info;
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Decoupled look-back by one full warp: the exclusive prefix of `tile` over the
// per-tile values published in lb[] (one 64-bit entry per tile).  Lane l reads
// predecessor (base - l), so each round trip inspects 32 tiles; entries are
// consumed nearest-first up to the first inclusive one.  Tiles below 0 count
// as an inclusive zero.  Bounded: after kLimit empty rounds the status is
// latched and the partial prefix returned.  All lanes return the same value.
template <uint64_t kLimit = kSpinLimit>
__device__ __forceinline__ uint32_t warp_lookback(const unsigned long long* lb, uint32_t tile,
                                                  uint32_t tag, FrameState* st, uint32_t site)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t tg = tag & 0x3FFFFFFFu;
    uint32_t prefix = 0;
    int base = (int)tile - 1;
    uint64_t spins = 0;
    while (base >= 0) {
        const int j = base - (int)lane;
        bool ready = true, incl = true;
        uint32_t val = 0;
        if (j >= 0) {
            const unsigned long long e = ld_lb_u64(lb + j);
            const unsigned long long flag = (e >> 32) & 3ull;
            ready = ((uint32_t)(e >> 34) == tg) && flag != 0;
            incl = flag == kFlagIncl;
            val = (uint32_t)e;
        }
        const uint32_t nr = __ballot_sync(0xffffffffu, !ready);
        const uint32_t first_nr = nr ? (uint32_t)(__ffs(nr) - 1) : 32u;
        const uint32_t usable = first_nr == 32u ? 0xffffffffu : ((1u << first_nr) - 1u);
        const uint32_t inc = __ballot_sync(0xffffffffu, ready && incl) & usable;
        const uint32_t take = inc ? (uint32_t)__ffs(inc) : first_nr;   // lanes consumed
        prefix += warp_sum_u32(lane < take ? val : 0u);
        if (inc) break;
        if (take == 0) {
            if (++spins > kLimit) {
                set_status(st, kErrTimeout, site);
                break;
            }
            __nanosleep(20);
        }
        base -= (int)take;
    }
    return prefix;
}

// ---------------------------------------------------------------------
// host launchers (one per kernel family)
// ---------------------------------------------------------------------
// Launch with programmatic stream serialisation (see grid_dep_wait).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Resident blocks per SM of each persistent / grid-stride kernel (occupancy API).
int occ_filter_pred();
int occ_filter_anc();
int occ_compact();
int occ_project();
int occ_scatter();
int occ_segsort();

// All launchers enqueue on `s` and read counts (M, N_P) from device memory,
// so a frame needs no host synchronisation.
// Zeroes the frame's counters: FrameState, the per-tile pair counts tile_cnt and
// the per-compaction-tile selection counts sel_cnt.
void launch_frame_begin(FrameState* st, uint32_t* tile_cnt, int n_tiles, uint32_t* sel_cnt, int n_sel_tiles,
                        cudaStream_t s);
void launch_filter_pred(const DevTree& t, const DevCamera& cam, uint32_t* pbits, FrameState* count_st, int blocks,
                        cudaStream_t s);
// The per-128-node boxes of the centres (t.cbox) from t.mu.
void launch_chunk_boxes(const DevTree& t, int sms, cudaStream_t s);
// Also adds each word's selected nodes to sel_cnt[word / kSelTileWords].
void launch_filter_anc(const DevTree& t, const uint32_t* pbits, uint32_t* selbits, uint32_t* sel_cnt,
                       int blocks, cudaStream_t s);
// Writes at most cap ids; more survivors latch FGS_ERR_CAPACITY and M = cap.
// Failure-detection probe: one warp waits through warp_lookback on an entry of
// lb that nothing publishes (a tag no frame uses), gives up after kProbeSpins
// empty rounds and latches kErrTimeout with site kProbeSite.
constexpr uint64_t kProbeSpins = 4096;
constexpr uint32_t kProbeSite = 0x7F0u;
void launch_wait_probe(const unsigned long long* lb, FrameState* st, cudaStream_t s);
void launch_compact(const uint32_t* selbits, uint32_t n_words, uint32_t* sel, uint32_t cap,
                    unsigned long long* lookback, FrameState* st, int blocks, cudaStream_t s);
// The same result from the Ancestor filter's per-tile counts (one block a tile).
void launch_compact_counted(const uint32_t* selbits, uint32_t n_words, uint32_t* sel, uint32_t cap,
                            const uint32_t* sel_cnt, FrameState* st, cudaStream_t s);
// Projection (splat records, footprints) and the per-tile pair counts
// tile_cnt[tiles] (zeroed by launch_frame_begin).
void launch_project(const DevTree& t, const DevCamera& cam, const uint32_t* sel, float* splat,
                    uint4* foot, uint32_t* tile_cnt, FrameState* st, int blocks, cudaStream_t s);
// Tile ranges (clamped to cap), scatter cursors (in tile_cnt), N_P and the list
// of tiles with more than kSegSmall pairs (large[], their number in
// FrameState::tickets[kTicketLarge]); lookback holds
// tile_scan_lookback_entries(n_tiles) entries; blocks at most the resident
// capacity (sms * occ_tile_scan()).
void launch_tile_scan(uint32_t* tile_cnt, uint2* ranges, uint32_t n_tiles, uint32_t* large,
                      unsigned long long cap, unsigned long long* lookback, FrameState* st, int blocks,
                      cudaStream_t s);
int occ_tile_scan();
// Look-back entries the tile scan needs for n_tiles tiles.
inline size_t tile_scan_lookback_entries(size_t n_tiles) { return n_tiles / 2048 + 2; }
// Every pair into its tile's bucket of items[] (depth bits << 32 | rank).
void launch_scatter(const DevCamera& cam, const uint4* foot, uint32_t* cursor, unsigned long long* items,
                    unsigned long long cap, FrameState* st, int blocks, cudaStream_t s);
void launch_scatter_batch(const DevCamera* cams, const uint32_t* tile_base, uint32_t n_pad,
                          const uint32_t* sel, const uint4* foot, uint32_t* cursor,
                          unsigned long long* items, unsigned long long cap, FrameState* st, int blocks,
                          cudaStream_t s);
// Sorts every tile's bucket of items[] into keys_out (tile << 32 | depth bits)
// and vals_out (rank), in place of the bucket's slots.
void launch_segsort(const uint2* ranges, uint32_t n_tiles, const uint32_t* large, unsigned long long* items,
                    unsigned long long* keys_out, uint32_t* vals_out, FrameState* st, int blocks,
                    cudaStream_t s);
// count: use the counting variant (fills FrameState::blend_* work counters)
void launch_blend(const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                  const float* splat, float* rgb, float* T, uint2* keep, FrameState* st, bool count,
                  cudaStream_t s);
void launch_blend_kpc(const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                      const float* splat, float* kpc, float* G, FrameState* st, cudaStream_t s);

void launch_eval_exp(const float* x, float* y, uint64_t n, cudaStream_t s);
void launch_batch_front(const DevTree& t, const DevCamera* cams, int V, uint32_t total_tiles,
                        const uint32_t* tile_base, uint32_t* pbits, uint32_t* selbits, uint32_t* sel,
                        uint32_t sel_cap, float* splat, uint4* foot, uint32_t* tile_cnt, uint32_t* large,
                        unsigned long long* items, unsigned long long* keys, uint32_t* vals,
                        unsigned long long cap, unsigned long long* lb_compact, unsigned long long* lb_scan, uint2* ranges,
                        FrameState* st, int sms, cudaStream_t s);
void launch_batch_blend(const DevCamera* cams, int V, uint32_t total_tiles, const uint32_t* tile_base,
                        const unsigned long long* img_off, const uint2* ranges, const uint32_t* vals,
                        const float* splat, float* rgb, float* T, FrameState* st, cudaStream_t s);
void launch_prep_params(const DevTree& t, const float* mu, const float* log_scale, const float* quat,
                        const float* logit, const float* sh, int blocks, cudaStream_t s);
// keep: per-pixel {final T, stop} buffer; kept: the last forward filled it
// (FGS_RENDER_KEEP), otherwise the blend backward recomputes it there.
void launch_backward(const DevTree& t, const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                     const float* splat, uint2* keep, bool kept, const uint32_t* sel, const float* dL_drgb,
                     float* gsplat,
                     const float* const params[5], float* const grads[5], bool accumulate, int proj_blocks,
                     FrameState* st, cudaStream_t s);
void launch_levelwise_step(const DevTree& t, const DevCamera& cam, const uint32_t* child_start,
                           const uint32_t* children, const uint32_t* frontier, uint32_t n_front,
                           uint32_t* next, uint32_t* n_next, uint32_t* selbits, cudaStream_t s);

}  // namespace fgs
