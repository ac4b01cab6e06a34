// Warp-cooperative enumeration of Gaussian-tile pairs, shared by the
// projection (per-tile pair counts) and the key scatter, single-view and
// batched.
#pragma once

#include "fgs_internal.cuh"

namespace fgs {

// Lane L of a full warp holds Gaussian L's footprint: rect_x = x0 | x1 << 16,
// rect_y = y0 | y1 << 16 (half-open tile ranges), its pair count cnt
// (= (x1 - x0)(y1 - y0), 0 if it emits nothing), the width of its view's tile
// grid tiles_x, that view's first tile id tile_base, and two payload words.
// The warp's pairs are numbered in Gaussian order, row-major within a
// rectangle, and handed out 32 per round: lane l of the round starting at q0
// gets pair q0 + l.
struct WarpPairs {
    uint32_t incl, excl, wtot, rect_x, rect_y, tiles_x, tile_base, pa, pb;

    __device__ __forceinline__ WarpPairs(uint32_t cnt, uint32_t rx, uint32_t ry, uint32_t tx, uint32_t tb,
                                         uint32_t a, uint32_t b)
        : rect_x(rx), rect_y(ry), tiles_x(tx), tile_base(tb), pa(a), pb(b)
    {
        const uint32_t lane = threadIdx.x & 31;
        incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t up = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += up;
        }
        wtot = __shfl_sync(0xffffffffu, incl, 31);
        excl = incl - cnt;
    }

    // This lane's pair of the round starting at q0: whether it exists, its
    // tile (0xFFFFFFFF if not) and the owner's payload.  All lanes must call it.
    __device__ __forceinline__ bool get(uint32_t q0, uint32_t& tile, uint32_t& o_pa, uint32_t& o_pb) const
    {
        const uint32_t lane = threadIdx.x & 31;
        const uint32_t q = q0 + lane;
        // owner of pair q: the first lane whose inclusive count exceeds q
        uint32_t lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t probe = __shfl_sync(0xffffffffu, incl, lo + step - 1);
            if (probe <= q) lo += step;
        }
        lo = lo < 31u ? lo : 31u;
        const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, lo);
        const uint32_t o_rx = __shfl_sync(0xffffffffu, rect_x, lo);
        const uint32_t o_ry = __shfl_sync(0xffffffffu, rect_y, lo);
        const uint32_t o_tx = __shfl_sync(0xffffffffu, tiles_x, lo);
        const uint32_t o_tb = __shfl_sync(0xffffffffu, tile_base, lo);
        o_pa = __shfl_sync(0xffffffffu, pa, lo);
        o_pb = __shfl_sync(0xffffffffu, pb, lo);
        tile = 0xFFFFFFFFu;
        if (q >= wtot) return false;
        const uint32_t x0 = o_rx & 0xFFFFu, rw = (o_rx >> 16) - x0;
        const uint32_t y0 = o_ry & 0xFFFFu;
        const uint32_t k = q - o_excl;
        tile = o_tb + (y0 + k / rw) * o_tx + (x0 + k % rw);
        return true;
    }
};

// Pair counts above which the projection's (and the scatter's) warp enumerates
// a Gaussian's pairs with all its lanes instead of in its rounds: a footprint
// of thousands of tiles would otherwise keep one warp walking hundreds of rounds
// alone while the rest of the grid has finished.
constexpr uint32_t kWarpWidePairs = 128;

// The lanes of a round that share a tile form one group; its lowest lane is
// the leader.  Returns the group mask.
__device__ __forceinline__ uint32_t tile_group(bool valid, uint32_t tile)
{
    const uint32_t grp = __match_any_sync(0xffffffffu, tile);
    return valid ? grp : 0u;
}

// Count every pair of a warp's Gaussians into tile_cnt: one reduction per tile
// and round (the lanes of a round that share a tile add together).  A Gaussian
// with more than kWarpWidePairs pairs is counted first by all 32 lanes, one tile of
// its rectangle a lane and step (all distinct tiles, so plain reductions).
__device__ __forceinline__ void warp_count_pairs(uint32_t cnt, uint32_t rect_x, uint32_t rect_y,
                                                 uint32_t tiles_x, uint32_t tile_base,
                                                 uint32_t* __restrict__ tile_cnt)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t wide = __ballot_sync(0xffffffffu, cnt > kWarpWidePairs);
    while (wide) {
        const uint32_t b = (uint32_t)__ffs(wide) - 1u;
        wide &= wide - 1u;
        const uint32_t n = __shfl_sync(0xffffffffu, cnt, b);
        const uint32_t rx = __shfl_sync(0xffffffffu, rect_x, b), ry = __shfl_sync(0xffffffffu, rect_y, b);
        const uint32_t tx = __shfl_sync(0xffffffffu, tiles_x, b), tb = __shfl_sync(0xffffffffu, tile_base, b);
        const uint32_t x0 = rx & 0xFFFFu, rw = (rx >> 16) - x0, y0 = ry & 0xFFFFu;
        for (uint32_t k = lane; k < n; k += 32) atomicAdd(tile_cnt + tb + (y0 + k / rw) * tx + (x0 + k % rw), 1u);
    }
    if (cnt > kWarpWidePairs) cnt = 0;
    if (__ballot_sync(0xffffffffu, cnt != 0) == 0u) return;
    const WarpPairs wp(cnt, rect_x, rect_y, tiles_x, tile_base, 0u, 0u);
    for (uint32_t q0 = 0; q0 < wp.wtot; q0 += 32) {
        uint32_t tile, a, b;
        const bool valid = wp.get(q0, tile, a, b);
        const uint32_t grp = tile_group(valid, tile);
        if (grp && lane == (uint32_t)(__ffs(grp) - 1)) atomicAdd(tile_cnt + tile, (uint32_t)__popc(grp));
    }
}

// Tile of pair k of footprint f (row-major in its rectangle).
__device__ __forceinline__ uint32_t rect_tile(const uint4& f, uint32_t k, uint32_t tiles_x, uint32_t tile_base)
{
    const uint32_t x0 = f.x & 0xFFFFu, rw = (f.x >> 16) - x0;
    const uint32_t y0 = f.y & 0xFFFFu;
    return tile_base + (y0 + k / rw) * tiles_x + (x0 + k % rw);
}

}  // namespace fgs
