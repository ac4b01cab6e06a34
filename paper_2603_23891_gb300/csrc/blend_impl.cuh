// Per-tile blending machinery shared by the single-view and the batched blend
// kernels (see blend.cu for the design).
#pragma once

#include "fgs_internal.cuh"

namespace fgs {
namespace blendk {




constexpr int kChunk = 256;
constexpr int kValsSlots = kChunk + 8;     // aligned superset of one chunk

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// 1D bulk copy global -> shared; src, dst 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <bool kKpc>
struct BlendSmem {
    uint32_t vals[kValsSlots];
    float4 g0[kChunk];          // u, v, A', B'  (power coefficients, see power_of)
    float4 g1[kChunk];          // C', lthr, alpha0, depth
    float4 g2[kChunk];          // r, g, b, radius
    uint32_t wmask[kChunk];     // bit w: warp w's pixels can reach the skip threshold
    alignas(16) uint16_t wlist[8][kChunk];  // per-warp list of chunk entries, in order
    float kpc_w[kKpc ? 8 : 1][kKpc ? kChunk : 1];   // per-warp partial KPC (Eq. 5)
    uint64_t bar;
    int timed_out;
};

// Entries of a half-block list whose powers a walk tests before applying hits.
constexpr int kGroup = 32;

// The Gaussian's exponent at offset (dx, dy) = (u - px, v - py):
// -1/2 (A dx^2 + 2 B dx dy + C dy^2) = (A' dx + B' dy) dx + (C' dy) dy with the
// per-Gaussian coefficients A' = -A/2, B' = -B, C' = -C/2, evaluated with two
// fused multiply-adds in this order (the reading both sides share).
__device__ __forceinline__ float power_of(float Ah, float Bn, float Ch, float dx, float dy)
{
    return ff(ff(Ah, dx, fm(Bn, dy)), dx, fm(fm(Ch, dy), dy));
}

// Shared-memory copy of a splat record's first two float4 (u, v, A, B),
// (C, lthr, alpha0, depth) with the conic replaced by the power coefficients.
__device__ __forceinline__ void put_coeffs(float4& d0, float4& d1, float4 a, float4 b)
{
    d0 = make_float4(a.x, a.y, fm(-0.5f, a.z), -a.w);
    d1 = make_float4(fm(-0.5f, b.x), b.y, b.z, b.w);
}

// Bring chunk [s0, e0) of the sorted values into shared memory with one TMA bulk
// copy of the 16-byte aligned superset [s0 & ~3, (e0 + 3) & ~3).  Returns the
// offset of s0 inside the staged copy.  Called by all threads; thread 0 issues
// the copy and waits on the mbarrier (bounded).  If the wait gives up, the
// status FGS_ERR_TIMEOUT is latched and the callers leave the tile; the copy may
// still be in flight into the block's shared memory as the block exits, so
// after such a timeout neither the frame's output nor the context can be
// trusted (the caller must destroy the context).
__device__ __forceinline__ uint32_t stage_vals(uint32_t* dst, uint64_t* bar, int* timed_out,
                                               const uint32_t* vals, uint32_t s0, uint32_t e0,
                                               uint32_t& phase, FrameState* st)
{
    const uint32_t a0 = s0 & ~3u;
    const uint32_t a1 = (e0 + 3u) & ~3u;
    const uint32_t bytes = (a1 - a0) * 4u;
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, bytes);
        tma_bulk_g2s(dst, vals + a0, bytes, bar);
        uint64_t spins = 0;
        while (!mbar_try_wait(bar, phase)) {
            if (++spins > kSpinLimit) {
                *timed_out = 1;
                set_status(st, kErrTimeout, 0x500u);
                break;
            }
        }
    }
    phase ^= 1u;
    __syncthreads();
    return s0 - a0;
}

// Warps of a CTA cover ww x wh pixel blocks of the tile, ww = 1 << warp_shift
// (8 or 4), wh = 32 / ww, tile_w / ww of them across; (tx0, ty0) is the tile's
// first pixel.
__device__ __forceinline__ void warp_origin(const DevCamera& cam, int32_t tx0, int32_t ty0, uint32_t w,
                                            int32_t& x0, int32_t& y0)
{
    const uint32_t sh = (uint32_t)(cam.tile_shift_x - cam.warp_shift);   // log2(warps per row)
    x0 = tx0 + (int32_t)((w & ((1u << sh) - 1u)) << cam.warp_shift);
    y0 = ty0 + (int32_t)((w >> sh) << (5 - cam.warp_shift));
}

// Which warps of the tile may hold a pixel whose binary32 power reaches the
// Gaussian's skip threshold lthr.  Exactly, power >= lthr is the ellipse
// d^T Q d <= s with Q = [[A, B], [B, C]] and s = -2 lthr, whose bounding box has
// half-widths sqrt(s C / det Q) and sqrt(s A / det Q).  Margins, for
// cond(Q) < 1e4 (cond(Q) <= tr^2 / det; beyond that, or for a singular Q, every
// warp keeps the Gaussian):
//  * the binary32 power (offsets rounded, three products, two fused
//    multiply-adds) is within 11 * 2^-24 * cond(Q) < 0.7% of the exact form at
//    the exact offsets, so a pixel passing the test lies in the ellipse of
//    s' = 1.05 s + 1e-4;
//  * det Q computed in binary32 loses at most 2^-24 cond(Q) / 2 < 3e-4
//    relative, so the computed half-widths are within 2e-4 relative of the
//    exact ones for s' (the 5% in s leaves 2% of the half-width spare);
//  * the box is further widened by 0.1% and 0.01 px for the roundings of
//    u - tx0, v - ty0 and of the bounds below.
// A warp left out of the mask would have skipped the Gaussian at every one of
// its pixels.  Warp column c spans pixel centres tx0 + ww c + [0.5, ww - 0.5],
// row r spans ty0 + wh r + [0.5, wh - 0.5]; the mask is the block of columns x
// rows the box meets.  (A one-pixel margin here listed 28% more entries for the
// few-pixel Gaussians of far LoD levels; an exact ellipse-rectangle test per
// warp removed only 4% more and cost more than it saved.)
__device__ __forceinline__ uint32_t warp_mask(const DevCamera& cam, int32_t tx0, int32_t ty0, float u,
                                              float v, float A, float B, float C, float lthr)
{
    if (!(lthr <= 0.0f)) return 0u;             // alpha0 < 1/255: no pixel can pass
    const float det = A * C - B * B;
    const float tr = A + C;
    if (!(det > 0.0f) || tr * tr > 1e4f * det) return 0xFFu;
    const float sq = fmaf(-2.1f, lthr, 1e-4f);  // 1.05 * (-2 lthr) + 1e-4
    const float ex = fmaf(sqrtf(sq * C / det), 1.001f, 0.01f);
    const float ey = fmaf(sqrtf(sq * A / det), 1.001f, 0.01f);
    const int32_t sh = cam.tile_shift_x - cam.warp_shift;   // log2(warps per tile row)
    const int32_t ncol = 1 << sh, nrow = 8 >> sh;
    const float ww = (float)(1 << cam.warp_shift), wh = (float)(32 >> cam.warp_shift);
    const float iww = 1.0f / ww, iwh = 1.0f / wh;            // exact: powers of two
    const float ux = u - (float)tx0, vy = v - (float)ty0;
    const int32_t c_lo = max(0, (int32_t)ceilf((ux - ex - (ww - 0.5f)) * iww));
    const int32_t c_hi = min(ncol - 1, (int32_t)floorf((ux + ex - 0.5f) * iww));
    const int32_t r_lo = max(0, (int32_t)ceilf((vy - ey - (wh - 0.5f)) * iwh));
    const int32_t r_hi = min(nrow - 1, (int32_t)floorf((vy + ey - 0.5f) * iwh));
    if (c_lo > c_hi || r_lo > r_hi) return 0u;
    const uint32_t cols = ((2u << c_hi) - 1u) & ~((1u << c_lo) - 1u);
    uint32_t mask = 0;
    for (int32_t r = r_lo; r <= r_hi; ++r) mask |= cols << (r << sh);
    return mask;
}


// The KPC pre-render of one tile (the CTA's; Eq. 5-6): the forward walk with
// per-warp lists, one entry at a time, every lane computing power and (when any
// lane of the warp can apply the Gaussian) alpha and T', selected per lane; the
// applied alpha * T is reduced across the warp per entry and over the warps per
// pair.  Writes kpc_out[pair] and the tile's mean KPC G_out[tile] (NaN for a
// tile without pairs).  No image is written.
__device__ __forceinline__ void blend_tile_kpc(const DevCamera& cam, uint32_t tile, BlendSmem<true>& S,
                                               double* s_red, const uint2* __restrict__ ranges,
                                               const uint32_t* __restrict__ vals,
                                               const float* __restrict__ splat,
                                               float* __restrict__ kpc_out, float* __restrict__ G_out,
                                               FrameState* st)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t tx0 = (int32_t)(tile % (uint32_t)cam.tiles_x) * cam.tile_w;
    const int32_t ty0 = (int32_t)(tile / (uint32_t)cam.tiles_x) * cam.tile_h;
    int32_t wx0, wy0;
    warp_origin(cam, tx0, ty0, warp, wx0, wy0);
    const int32_t x = wx0 + (int32_t)(lane & ((1u << cam.warp_shift) - 1u));
    const int32_t y = wy0 + (int32_t)(lane >> cam.warp_shift);
    const bool inside = x < cam.width && y < cam.height;
    const float px = fa((float)x, 0.5f), py = fa((float)y, 0.5f);
    const uint2 rg = ranges[tile];
    const uint32_t M = st->M;
    const uint32_t s = rg.x, e = rg.y;

    if (tid == 0) {
        mbar_init(&S.bar, 1);
        S.timed_out = 0;
    }
    __syncthreads();

    float T = 1.0f;
    bool done = !inside;
    uint32_t phase = 0;
    double kpc_acc = 0.0;      // this thread's share of the tile's KPC sum (fixed order)

    for (uint32_t s0 = s; s0 < e; s0 += kChunk) {
        const uint32_t e0 = min(e, s0 + kChunk);
        const uint32_t cnt = e0 - s0;
        const uint32_t off = stage_vals(S.vals, &S.bar, &S.timed_out, vals, s0, e0, phase, st);
        if (S.timed_out) break;
        if (tid < cnt) {
            uint32_t m = S.vals[off + tid];
            if (m >= M) m = 0;      // only after a failed sort (status already latched)
            const float4* g = reinterpret_cast<const float4*>(splat + (size_t)m * kSplatStride);
            const float4 a = __ldg(g), b = __ldg(g + 1);
            put_coeffs(S.g0[tid], S.g1[tid], a, b);
            S.wmask[tid] = warp_mask(cam, tx0, ty0, a.x, a.y, a.z, a.w, b.x, b.y);
        }
        __syncthreads();
        // this warp's ordered list of the chunk entries that can reach its pixels
        uint32_t wcnt = 0;
        for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool mine = j < cnt && ((S.wmask[j] >> warp) & 1u);
            const uint32_t b = __ballot_sync(0xffffffffu, mine);
            if (mine) S.wlist[warp][wcnt + __popc(b & ((1u << lane) - 1u))] = (uint16_t)j;
            wcnt += __popc(b);
        }
        __syncwarp();
        for (uint32_t i = 0; i < wcnt; ++i) {
            const uint32_t j = S.wlist[warp][i];
            float w = 0.0f;
            const float4 g0 = S.g0[j];
            const float4 g1 = S.g1[j];
            const float power = power_of(g0.z, g0.w, g1.x, fs(g0.x, px), fs(g0.y, py));
            const bool hit = !done && !(power > 0.0f || power < g1.y);
            if (__any_sync(0xffffffffu, hit)) {
                float alpha = fm(g1.z, exp_nonpos(fminf(power, 0.0f)));
                alpha = alpha < 0.99f ? alpha : 0.99f;
                const float Tn = fm(T, fs(1.0f, alpha));
                const bool stop = hit && Tn < 0.0001f;     // stop before adding this Gaussian
                const bool apply = hit && !stop;
                w = apply ? alpha * T : 0.0f;
                T = apply ? Tn : T;
                done = done || stop;
            }
            // Eq. 5: sum of alpha * T over the warp's pixels for this pair
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if (lane == 0) S.kpc_w[warp][j] = w;
        }
        __syncthreads();
        if (tid < cnt) {
            const uint32_t msk = S.wmask[tid];
            float k = 0.0f;
#pragma unroll
            for (int w8 = 0; w8 < 8; ++w8)
                if ((msk >> w8) & 1u) k += S.kpc_w[w8][tid];
            kpc_out[s0 + tid] = k;
            kpc_acc += (double)k;
        }
        __syncthreads();
    }
    // Eq. 6: G = mean KPC over the tile's pairs; fixed-order block reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kpc_acc += __shfl_xor_sync(0xffffffffu, kpc_acc, o);
    if (lane == 0) s_red[warp] = kpc_acc;
    __syncthreads();
    if (tid == 0) {
        const uint32_t n = e - s;
        double sum = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) sum += s_red[w8];
        G_out[tile] = n > 0 ? (float)(sum / (double)n) : __int_as_float(0x7fc00000);
    }
}

// ---------------------------------------------------------------------------
// Half-warp culling: the forward's walk over 4x4-pixel half-blocks
// ---------------------------------------------------------------------------
// Each warp's 32 pixels are two 4x4 half-blocks (lanes 0-15 and 16-31), side by
// side for 8x4 warps, stacked for 4x8 warps; a tile holds 16 of them.  Every
// half-block has its own ordered list of the chunk's Gaussians whose threshold
// box meets it, so a Gaussian a few pixels across is tested by the 16 lanes of
// each half it can reach instead of by all 32 lanes of each warp (about 25%
// fewer lockstep steps on far LoD levels).  Both halves of a warp walk their
// own lists in lockstep.
constexpr int kHalfBlocks = 16;

struct HalfSmem {
    uint32_t vals[2][kValsSlots];               // two chunks of values: the walked one, the next
    float4 g0[kChunk];                          // u, v, A', B'
    float4 g1[kChunk];                          // C', lthr, alpha0, depth
    uint16_t hmask[kChunk];                     // bit b: half-block b may hold a pixel reaching lthr
    alignas(16) uint8_t hl[kHalfBlocks][kChunk];   // per half-block ordered list of chunk slots
    float pw[8][kGroup][32];                    // each lane's power per group entry
    float4 grp[8][2][kGroup];                   // alpha0, r, g, b per half and group entry
    uint64_t bar[2];                            // completion of each values buffer's copy
    int timed_out;
};

// Thread 0: start the TMA bulk copy of chunk [s0, e0) of the sorted values into
// dst (the 16-byte aligned superset [s0 & ~3, (e0 + 3) & ~3)), completing on bar.
__device__ __forceinline__ void stage_issue(uint32_t* dst, uint64_t* bar, const uint32_t* vals, uint32_t s0,
                                            uint32_t e0)
{
    const uint32_t a0 = s0 & ~3u;
    const uint32_t a1 = (e0 + 3u) & ~3u;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (a1 - a0) * 4u);
    tma_bulk_g2s(dst, vals + a0, (a1 - a0) * 4u, bar);
}

// Thread 0: wait for the copy on bar to complete phase `phase` (bounded: on
// giving up FGS_ERR_TIMEOUT is latched and *timed_out set, as in stage_vals).
__device__ __forceinline__ void stage_wait(uint64_t* bar, uint32_t phase, int* timed_out, FrameState* st)
{
    uint64_t spins = 0;
    while (!mbar_try_wait(bar, phase)) {
        if (++spins > kSpinLimit) {
            *timed_out = 1;
            set_status(st, kErrTimeout, 0x500u);
            break;
        }
    }
}

// Half-blocks of the tile (grid of tile_w / 4 x tile_h / 4, row-major bits) that
// the Gaussian's threshold box meets; the box and its margins are warp_mask's.
__device__ __forceinline__ uint32_t half_mask(const DevCamera& cam, int32_t tx0, int32_t ty0, float u,
                                              float v, float A, float B, float C, float lthr)
{
    if (!(lthr <= 0.0f)) return 0u;
    const float det = A * C - B * B;
    const float tr = A + C;
    if (!(det > 0.0f) || tr * tr > 1e4f * det) return 0xFFFFu;
    const float sq = fmaf(-2.1f, lthr, 1e-4f);
    const float ex = fmaf(sqrtf(sq * C / det), 1.001f, 0.01f);
    const float ey = fmaf(sqrtf(sq * A / det), 1.001f, 0.01f);
    const int32_t sh = cam.tile_shift_x - 2;                 // log2(half-block columns)
    const int32_t ncol = 1 << sh, nrow = kHalfBlocks >> sh;
    const float ux = u - (float)tx0, vy = v - (float)ty0;
    const int32_t c_lo = max(0, (int32_t)ceilf((ux - ex - 3.5f) * 0.25f));
    const int32_t c_hi = min(ncol - 1, (int32_t)floorf((ux + ex - 0.5f) * 0.25f));
    const int32_t r_lo = max(0, (int32_t)ceilf((vy - ey - 3.5f) * 0.25f));
    const int32_t r_hi = min(nrow - 1, (int32_t)floorf((vy + ey - 0.5f) * 0.25f));
    if (c_lo > c_hi || r_lo > r_hi) return 0u;
    const uint32_t cols = ((2u << c_hi) - 1u) & ~((1u << c_lo) - 1u);
    uint32_t mask = 0;
    for (int32_t r = r_lo; r <= r_hi; ++r) mask |= cols << (r << sh);
    return mask;
}

// Phase 1 of the group walk: this lane's binary32 power for each entry of its
// half-block's group (the list wl of 8-bit chunk slots), parked in pw[e][lane],
// and the bit mask of the entries whose power passes both skip tests.  The
// list is read four entries at a time; the warp-uniform bound ngw covers both
// halves' groups and bits past this half's own ng are cleared.  Any 8-bit slot
// indexes the chunk arrays, so entries read past a list's end are harmless and
// masked.
__device__ __forceinline__ uint32_t half_group_tests(const float4* __restrict__ g0s,
                                                     const float4* __restrict__ g1s, const uint8_t* wl,
                                                     uint32_t ngw, uint32_t ng, float px, float py,
                                                     float (*pw)[32], uint32_t lane)
{
    const uint32_t* wl4 = reinterpret_cast<const uint32_t*>(wl);
    uint32_t hits = 0;
    for (uint32_t e = 0; e < ngw; e += 4) {
        const uint32_t jj = wl4[e >> 2];
        const uint32_t jx[4] = {jj & 0xffu, (jj >> 8) & 0xffu, (jj >> 16) & 0xffu, jj >> 24};
        uint32_t nib = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 a = g0s[jx[k]];
            const float4 b = g1s[jx[k]];
            const float power = power_of(a.z, a.w, b.x, fs(a.x, px), fs(a.y, py));
            pw[e + k][lane] = power;
            nib |= (uint32_t)!(power > 0.0f || power < b.y) << k;
        }
        hits |= nib << e;
    }
    return ng >= 32u ? hits : hits & ((1u << ng) - 1u);
}

// Blend one image tile with half-block lists (the forward without KPC).
// `tile` is the tile in the camera's grid; `gtile` indexes ranges (the same
// for one view; the batch's global tile id).  rgb / Tout are the camera's own
// image planes.  With kKeep, keep_out receives per pixel {final T bits, stop
// position}: the sorted-pair index of the Gaussian the pixel stopped at, or the
// tile's end if it did not stop; the differentiable form's backward walks each
// pixel from there.  kCount adds the work counters of FrameState (lockstep
// warp steps, evaluations, alpha applications, steps with an application).
template <bool kCount = false, bool kKeep = false>
__device__ __forceinline__ void blend_tile_half(const DevCamera& cam, uint32_t tile, uint32_t gtile,
                                                HalfSmem& H, const uint2* __restrict__ ranges,
                                                const uint32_t* __restrict__ vals,
                                                const float* __restrict__ splat, float* __restrict__ rgb,
                                                float* __restrict__ Tout, uint2* __restrict__ keep_out,
                                                FrameState* st)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t tx0 = (int32_t)(tile % (uint32_t)cam.tiles_x) * cam.tile_w;
    const int32_t ty0 = (int32_t)(tile / (uint32_t)cam.tiles_x) * cam.tile_h;
    int32_t wx0, wy0;
    warp_origin(cam, tx0, ty0, warp, wx0, wy0);
    const uint32_t half = lane >> 4, q = lane & 15u;
    const bool wide = cam.warp_shift == 3;       // 8x4 warps: halves side by side
    const int32_t x = wx0 + (int32_t)(q & 3u) + (wide ? 4 * (int32_t)half : 0);
    const int32_t y = wy0 + (int32_t)(q >> 2) + (wide ? 0 : 4 * (int32_t)half);
    const uint32_t hb = ((uint32_t)(y - ty0) >> 2 << (cam.tile_shift_x - 2)) | ((uint32_t)(x - tx0) >> 2);
    const uint32_t hb0 = __shfl_sync(0xffffffffu, hb, 0), hb1 = __shfl_sync(0xffffffffu, hb, 16);
    const bool inside = x < cam.width && y < cam.height;
    const float px = fa((float)x, 0.5f), py = fa((float)y, 0.5f);
    const uint2 rg = ranges[gtile];
    const uint32_t M = st->M;
    const uint32_t s = rg.x, e = rg.y;
    const uint32_t lt = (1u << lane) - 1u;

    if (tid == 0) {
        mbar_init(&H.bar[0], 1);
        mbar_init(&H.bar[1], 1);
        H.timed_out = 0;
        if (s < e) stage_issue(H.vals[0], &H.bar[0], vals, s, min(e, s + kChunk));
    }
    // every group entry's alpha0 and colour finite from the start
    static_assert(sizeof(H.grp) == 2 * 256 * sizeof(float4), "two float4 a thread");
    reinterpret_cast<float4*>(&H.grp[0][0][0])[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(&H.grp[0][0][0])[tid + 256] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    float T = 1.0f;
    float3 Cacc = make_float3(0.0f, 0.0f, 0.0f);
    bool done = !inside;
    // chunk k's values in buffer k & 1; the next chunk's copy is started once this
    // chunk's records are gathered, so it lands while the chunk is walked
    uint32_t phases = 0u;                       // bit i: the parity buffer i's copy completes next
    uint32_t k = 0;
    for (uint32_t s0 = s; s0 < e; s0 += kChunk, ++k) {
        const uint32_t e0 = min(e, s0 + kChunk);
        const uint32_t cnt = e0 - s0;
        const uint32_t bi = k & 1u;
        if (tid == 0) stage_wait(&H.bar[bi], (phases >> bi) & 1u, &H.timed_out, st);
        phases ^= 1u << bi;
        __syncthreads();
        if (H.timed_out) break;
        const uint32_t* cv = H.vals[bi];
        const uint32_t off = s0 - (s0 & ~3u);
        if (tid < cnt) {
            uint32_t m = cv[off + tid];
            if (m >= M) m = 0;      // only after a failed sort (status already latched)
            const float4* g = reinterpret_cast<const float4*>(splat + (size_t)m * kSplatStride);
            const float4 a = __ldg(g), b = __ldg(g + 1);
            put_coeffs(H.g0[tid], H.g1[tid], a, b);
            H.hmask[tid] = (uint16_t)half_mask(cam, tx0, ty0, a.x, a.y, a.z, a.w, b.x, b.y);
        }
        __syncthreads();
        // the other buffer's last reader (chunk k - 1's walk) has finished
        const bool more = s0 + kChunk < e;
        if (tid == 0 && more) stage_issue(H.vals[bi ^ 1u], &H.bar[bi ^ 1u], vals, s0 + kChunk, min(e, s0 + 2 * kChunk));
        // the ordered lists of this warp's two half-blocks
        uint32_t n0 = 0, n1 = 0;
        for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t hm = j < cnt ? (uint32_t)H.hmask[j] : 0u;
            const uint32_t b0 = __ballot_sync(0xffffffffu, (hm >> hb0) & 1u);
            const uint32_t b1 = __ballot_sync(0xffffffffu, (hm >> hb1) & 1u);
            if ((hm >> hb0) & 1u) H.hl[hb0][n0 + __popc(b0 & lt)] = (uint8_t)j;
            if ((hm >> hb1) & 1u) H.hl[hb1][n1 + __popc(b1 & lt)] = (uint8_t)j;
            n0 += __popc(b0);
            n1 += __popc(b1);
        }
        __syncwarp();
        const uint8_t* myl = H.hl[hb];
        uint32_t c_entries = 0, c_evals = 0, c_hits = 0, c_active = 0;
        float (*pw)[32] = H.pw[warp];
        const uint32_t nmax = max(n0, n1);
        for (uint32_t i0 = 0; i0 < nmax; i0 += kGroup) {
            if (__all_sync(0xffffffffu, done)) break;
            const uint32_t ngw = min((uint32_t)kGroup, nmax - i0);
            const uint32_t g0n = n0 > i0 ? min((uint32_t)kGroup, n0 - i0) : 0u;
            const uint32_t g1n = n1 > i0 ? min((uint32_t)kGroup, n1 - i0) : 0u;
            const uint32_t ng = half ? g1n : g0n;
            // colours of the group's entries, fetched now and stored after the tests
            uint32_t ja = 0, jb = 0;
            float4 ca = make_float4(0.f, 0.f, 0.f, 0.f), cb = ca;
            if (lane < g0n) {
                ja = H.hl[hb0][i0 + lane];
                uint32_t m = cv[off + ja];
                if (m >= M) m = 0;
                ca = __ldg(reinterpret_cast<const float4*>(splat + (size_t)m * kSplatStride) + 2);
            }
            if (lane < g1n) {
                jb = H.hl[hb1][i0 + lane];
                uint32_t m = cv[off + jb];
                if (m >= M) m = 0;
                cb = __ldg(reinterpret_cast<const float4*>(splat + (size_t)m * kSplatStride) + 2);
            }
            const bool done0 = done;
            uint32_t hits = half_group_tests(H.g0, H.g1, myl + i0, ngw, ng, px, py, pw, lane);
            if (done) hits = 0;
            if (lane < g0n) H.grp[warp][0][lane] = make_float4(H.g1[ja].z, ca.x, ca.y, ca.z);
            if (lane < g1n) H.grp[warp][1][lane] = make_float4(H.g1[jb].z, cb.x, cb.y, cb.z);
            __syncwarp();
            const float4* grp = H.grp[warp][half];
            uint32_t proc = 0, n_eval = ng;
            // as many rounds as the lane with most hits; a hit's power is at least
            // its skip threshold, -ln 255 - ln alpha0 >= -5.55, so exp_hit applies
            const uint32_t n_rounds = __reduce_max_sync(0xffffffffu, (uint32_t)__popc(hits));
            for (uint32_t round = 0; round < n_rounds; ++round) {
                // branch-free: a lane without a hit left (or whose application
                // stops) computes on entry 0 and adds nothing: w = 0 times a finite
                // colour (every group entry holds a real Gaussian's colour or the
                // zeros it was initialised with)
                const bool valid = hits != 0u;
                const uint32_t e = valid ? (uint32_t)(__ffs(hits) - 1) : 0u;
                hits &= hits - 1u;
                const float4 qv = grp[e];
                float alpha = fm(qv.x, exp_hit(pw[e][lane]));
                alpha = alpha < 0.99f ? alpha : 0.99f;
                const float Tn = fm(T, fs(1.0f, alpha));
                const bool stop = valid && Tn < 0.0001f;       // stop before adding this Gaussian
                const bool apply = valid && !(Tn < 0.0001f);
                const float w = apply ? alpha * T : 0.0f;
                Cacc.x = fmaf(qv.y, w, Cacc.x);
                Cacc.y = fmaf(qv.z, w, Cacc.y);
                Cacc.z = fmaf(qv.w, w, Cacc.z);
                if (kCount && valid) {
                    ++c_hits;
                    proc |= 1u << e;
                }
                if (kKeep && stop)
                    keep_out[(size_t)y * cam.width + x] = make_uint2(__float_as_uint(T), s0 + myl[i0 + e]);
                T = apply ? Tn : T;
                if (stop) {
                    done = true;
                    hits = 0;
                    n_eval = e + 1;
                }
            }
            __syncwarp();
            if (kCount) {
                c_entries += ngw;
                c_evals += warp_sum_u32(done0 ? 0u : n_eval);
                c_active += __popc(__reduce_or_sync(0xffffffffu, proc));
            }
        }
        if (kCount) {
            c_hits = warp_sum_u32(c_hits);
            if (lane == 0) {
                atomicAdd(&st->blend_entries, (unsigned long long)c_entries);
                atomicAdd(&st->blend_evals, (unsigned long long)c_evals);
                atomicAdd(&st->blend_hits, (unsigned long long)c_hits);
                atomicAdd(&st->blend_active, (unsigned long long)c_active);
            }
        }
        const int n_done = __syncthreads_count(done);
        if (n_done == (int)blockDim.x) {
            // a started copy must land before the block leaves
            if (more) {
                if (tid == 0) stage_wait(&H.bar[bi ^ 1u], (phases >> (bi ^ 1u)) & 1u, &H.timed_out, st);
                __syncthreads();
            }
            break;
        }
    }
    if (inside) {
        const size_t hw = (size_t)cam.width * cam.height;
        const size_t pix = (size_t)y * cam.width + x;
        if (rgb) {
            rgb[pix] = fmaf(T, cam.bg[0], Cacc.x);
            rgb[hw + pix] = fmaf(T, cam.bg[1], Cacc.y);
            rgb[2 * hw + pix] = fmaf(T, cam.bg[2], Cacc.z);
        }
        if (Tout) Tout[pix] = T;
        if (kKeep && !done) keep_out[pix] = make_uint2(__float_as_uint(T), e);   // did not stop
    }
}


}  // namespace blendk
}  // namespace fgs
