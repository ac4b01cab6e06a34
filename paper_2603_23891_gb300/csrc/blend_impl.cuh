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

// Per-warp scratch of the group walk (see blend_tile): each lane's binary32
// power for every entry of the group, and the entries' alpha0 and colour.
constexpr int kGroup = 32;
template <bool kUsed>
struct GroupSmem {
    float pw[kUsed ? 8 : 1][kUsed ? kGroup : 1][32];
    float4 grp[kUsed ? 8 : 1][kUsed ? kGroup : 1];   // alpha0, r, g, b
};

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

// Phase 1 of the group walk: this lane's binary32 power for each of the ng
// (<= kGroup) entries of the warp list wl (chunk slots), parked in pw[e][lane],
// and the bit mask of the entries whose power passes both skip tests.  The list
// is read four entries at a time; it must be padded with valid slots to a
// multiple of 4 (the padding's bits are cleared).
__device__ __forceinline__ uint32_t group_tests(const float4* __restrict__ g0s,
                                                const float4* __restrict__ g1s, const uint16_t* wl,
                                                uint32_t ng, float px, float py, float (*pw)[32],
                                                uint32_t lane)
{
    const uint2* wl4 = reinterpret_cast<const uint2*>(wl);
    uint32_t hits = 0;
    for (uint32_t e = 0; e < ng; e += 4) {
        const uint2 jj = wl4[e >> 2];
        const uint32_t jx[4] = {jj.x & 0xffffu, jj.x >> 16, jj.y & 0xffffu, jj.y >> 16};
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

// Bring chunk [s0, e0) of the sorted values into shared memory with one TMA bulk
// copy of the 16-byte aligned superset [s0 & ~3, (e0 + 3) & ~3).  Returns the
// offset of s0 inside the staged copy.  Called by all threads; thread 0 issues
// the copy and waits on the mbarrier (bounded).
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


// Blend one image tile (the CTA's).  `tile` is the tile in the camera's grid;
// `gtile` indexes ranges and G_out (the same for one view; the batch's global
// tile id).  rgb / Tout are the camera's own image planes.  With kKeep,
// keep_out receives per pixel {final T bits, stop position}: the sorted-pair
// index of the Gaussian the pixel stopped at, or the tile's end if it did not
// stop; the differentiable form's backward walks each pixel from there.
template <bool kKpc, bool kCount = false, bool kKeep = false>
__device__ __forceinline__ void blend_tile(const DevCamera& cam, uint32_t tile, uint32_t gtile,
                                           BlendSmem<kKpc>& S, GroupSmem<!kKpc>& Gs, double* s_red,
                                           const uint2* __restrict__ ranges,
                                           const uint32_t* __restrict__ vals,
                                           const float* __restrict__ splat, float* __restrict__ rgb,
                                           float* __restrict__ Tout, uint2* __restrict__ keep_out,
                                           float* __restrict__ kpc_out,
                                           float* __restrict__ G_out, FrameState* st)
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
    const uint2 rg = ranges[gtile];
    const uint32_t M = st->M;
    const uint32_t s = rg.x, e = rg.y;

    if (tid == 0) {
        mbar_init(&S.bar, 1);
        S.timed_out = 0;
    }
    __syncthreads();

    float T = 1.0f;
    float3 Cacc = make_float3(0.0f, 0.0f, 0.0f);
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
            S.g2[tid] = __ldg(g + 2);
            S.wmask[tid] = warp_mask(cam, tx0, ty0, a.x, a.y, a.z, a.w, b.x, b.y);
        }
        __syncthreads();
        // this warp's ordered list of the chunk entries that can reach its pixels,
        // padded with slot 0 to a multiple of 4 (group_tests reads 4 at a time)
        uint32_t wcnt = 0;
        for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool mine = j < cnt && ((S.wmask[j] >> warp) & 1u);
            const uint32_t b = __ballot_sync(0xffffffffu, mine);
            if (mine) S.wlist[warp][wcnt + __popc(b & ((1u << lane) - 1u))] = (uint16_t)j;
            wcnt += __popc(b);
        }
        if (wcnt + lane < ((wcnt + 3u) & ~3u)) S.wlist[warp][wcnt + lane] = 0;
        __syncwarp();
        uint32_t c_entries = 0, c_evals = 0, c_hits = 0, c_active = 0;
        if (kKpc) {
            // the KPC pass reduces alpha * T per entry across the warp: one entry at a time
            for (uint32_t i = 0; i < wcnt; ++i) {
                const uint32_t j = S.wlist[warp][i];
                float w = 0.0f;
                if (kCount) {
                    ++c_entries;
                    c_evals += __popc(__ballot_sync(0xffffffffu, !done));
                }
                // Branch-free evaluation: every lane computes power; if any lane of
                // the warp can apply the Gaussian, all compute alpha and T' and the
                // outcome is selected per lane.
                const float4 g0 = S.g0[j];
                const float4 g1 = S.g1[j];
                const float power = power_of(g0.z, g0.w, g1.x, fs(g0.x, px), fs(g0.y, py));
                const bool hit = !done && !(power > 0.0f || power < g1.y);
                if (__any_sync(0xffffffffu, hit)) {
                    if (kCount) {
                        c_hits += hit ? 1u : 0u;
                        ++c_active;
                    }
                    float alpha = fm(g1.z, exp_nonpos(fminf(power, 0.0f)));
                    alpha = alpha < 0.99f ? alpha : 0.99f;
                    const float Tn = fm(T, fs(1.0f, alpha));
                    const bool stop = hit && Tn < 0.0001f;     // stop before adding this Gaussian
                    const bool apply = hit && !stop;
                    if (kKeep && stop)
                        keep_out[(size_t)y * cam.width + x] = make_uint2(__float_as_uint(T), s0 + j);
                    const float4 g2 = S.g2[j];
                    w = apply ? alpha * T : 0.0f;
                    Cacc.x = fmaf(g2.x, w, Cacc.x);
                    Cacc.y = fmaf(g2.y, w, Cacc.y);
                    Cacc.z = fmaf(g2.z, w, Cacc.z);
                    T = apply ? Tn : T;
                    done = done || stop;
                }
                if (kKpc) {
                    // Eq. 5: sum of alpha * T over the warp's pixels for this pair
    #pragma unroll
                    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                    if (lane == 0) S.kpc_w[warp][j] = w;
                }
            }
        } else {
            // Groups of kGroup list entries.  Phase 1, in lockstep: every lane
            // tests every entry of the group, keeps a bit per entry it applies
            // and parks its binary32 power in shared memory.  Phase 2: every
            // lane applies its own entries in list order, the lanes of the warp
            // working on different entries at once, so the alpha / T / colour
            // work is spent only on pixels that apply.  A lane that stops drops
            // its remaining bits.  Each lane performs exactly the operations of
            // the one-entry-at-a-time walk, in the same order, so every
            // decision is unchanged.
            float (*pw)[32] = Gs.pw[warp];
            float4* grp = Gs.grp[warp];
            for (uint32_t i0 = 0; i0 < wcnt; i0 += kGroup) {
                if (__all_sync(0xffffffffu, done)) break;
                const uint32_t ng = min((uint32_t)kGroup, wcnt - i0);
                const bool done0 = done;
                uint32_t hits = group_tests(S.g0, S.g1, &S.wlist[warp][i0], ng, px, py, pw, lane);
                if (done) hits = 0;
                if (lane < ng) {
                    const uint32_t j = S.wlist[warp][i0 + lane];
                    const float4 c = S.g2[j];
                    grp[lane] = make_float4(S.g1[j].z, c.x, c.y, c.z);
                }
                __syncwarp();
                uint32_t proc = 0, n_eval = ng;
                while (__any_sync(0xffffffffu, hits != 0u)) {
                    if (hits) {
                        const uint32_t e = __ffs(hits) - 1;
                        hits &= hits - 1u;
                        const float4 q = grp[e];
                        float alpha = fm(q.x, exp_nonpos(pw[e][lane]));
                        alpha = alpha < 0.99f ? alpha : 0.99f;
                        const float Tn = fm(T, fs(1.0f, alpha));
                        if (kCount) {
                            ++c_hits;
                            proc |= 1u << e;
                        }
                        if (Tn < 0.0001f) {
                            done = true;                    // stop before adding this Gaussian
                            hits = 0;
                            n_eval = e + 1;
                            if (kKeep)
                                keep_out[(size_t)y * cam.width + x] =
                                    make_uint2(__float_as_uint(T), s0 + S.wlist[warp][i0 + e]);
                        } else {
                            const float w = alpha * T;
                            Cacc.x = fmaf(q.y, w, Cacc.x);
                            Cacc.y = fmaf(q.z, w, Cacc.y);
                            Cacc.z = fmaf(q.w, w, Cacc.z);
                            T = Tn;
                        }
                    }
                }
                __syncwarp();
                if (kCount) {
                    c_entries += ng;
                    c_evals += warp_sum_u32(done0 ? 0u : n_eval);
                    c_active += __popc(__reduce_or_sync(0xffffffffu, proc));
                }
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
        if (kKpc) {
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
        }
        const int n_done = __syncthreads_count(done);
        if (!kKpc && n_done == (int)blockDim.x) break;
    }
    if (inside && rgb) {
        const size_t hw = (size_t)cam.width * cam.height;
        const size_t pix = (size_t)y * cam.width + x;
        rgb[pix] = fmaf(T, cam.bg[0], Cacc.x);
        rgb[hw + pix] = fmaf(T, cam.bg[1], Cacc.y);
        rgb[2 * hw + pix] = fmaf(T, cam.bg[2], Cacc.z);
        if (Tout) Tout[pix] = T;
        if (kKeep && !done) keep_out[pix] = make_uint2(__float_as_uint(T), e);   // did not stop
    }
    if (kKpc) {
        // Eq. 6: G = mean KPC over the tile's pairs; fixed-order block reduction
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kpc_acc += __shfl_xor_sync(0xffffffffu, kpc_acc, o);
        if (lane == 0) s_red[warp] = kpc_acc;
        __syncthreads();
        if (tid == 0) {
            const uint32_t n = e - s;
            double sum = 0.0;
            for (int w8 = 0; w8 < 8; ++w8) sum += s_red[w8];
            G_out[gtile] = n > 0 ? (float)(sum / (double)n) : __int_as_float(0x7fc00000);
        }
    }
}


}  // namespace blendk
}  // namespace fgs
