// Traversal-free parallel filtering (§3.2) on sm_103a.
//
//  filter_pred        R&L filter: every node independently, P(n) = in-frustum and
//                     (leaf or R_2D = 3 sqrt(lambda_max) <= tau_R).  Streams the
//                     SoA centres with 16-byte loads; the covariance is read only
//                     for in-frustum internal nodes (a leaf passes on the frustum
//                     test alone).  Output: one bit per node.
//  filter_anc_compact Ancestor filter + stream compaction: a node with P walks its
//                     ancestor path AP (parent first, stopping at the first ancestor
//                     with P); survivors are compacted in ascending id order by warp
//                     ballots, a block scan and a decoupled look-back across tiles.
#include "fgs_internal.cuh"

namespace fgs {

__global__ void frame_begin_kernel(FrameState* st, uint2* ranges, int n_tiles)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        st->epoch = st->epoch + 1;
        st->M = 0;
        st->n_pairs = 0;
    }
    if (tid < 16) st->tickets[tid] = 0;
    for (int i = tid; i < kMaxSortPasses * 256; i += gridDim.x * blockDim.x)
        (&st->hist[0][0])[i] = 0;
    for (int i = tid; i < n_tiles; i += gridDim.x * blockDim.x) ranges[i] = make_uint2(0, 0);
}

void launch_frame_begin(FrameState* st, uint2* ranges, int n_tiles, cudaStream_t s)
{
    int blocks = (n_tiles + 255) / 256;
    blocks = blocks < 8 ? 8 : blocks;
    frame_begin_kernel<<<blocks, 256, 0, s>>>(st, ranges, n_tiles);
}

// ---------------------------------------------------------------------------
// R&L predicate: 4 consecutive nodes per thread, bits assembled per warp.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) filter_pred_kernel(DevTree t, DevCamera cam, uint32_t* pbits)
{
    const uint32_t n_chunks = t.n_pad >> 2;               // multiple of 32
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_chunks; i += stride) {
        const uint32_t n0 = i << 2;
        const float4 mx = __ldg(reinterpret_cast<const float4*>(t.mu) + i);
        const float4 my = __ldg(reinterpret_cast<const float4*>(t.mu + t.n_pad) + i);
        const float4 mz = __ldg(reinterpret_cast<const float4*>(t.mu + 2 * (size_t)t.n_pad) + i);
        const uint32_t leaf = (__ldg(t.leaf_bits + (i >> 3)) >> ((i & 7) << 2)) & 0xFu;
        const float xs[4] = {mx.x, mx.y, mx.z, mx.w};
        const float ys[4] = {my.x, my.y, my.z, my.w};
        const float zs[4] = {mz.x, mz.y, mz.z, mz.w};
        float vz[4], txtz[4], tytz[4];
        uint32_t inf = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float vx, vy;
            camera_space(cam, xs[k], ys[k], zs[k], vx, vy, vz[k]);
            txtz[k] = tytz[k] = 0.0f;
            const bool in = (n0 + k < t.n) && frustum_test(cam, vx, vy, vz[k], txtz[k], tytz[k]);
            inf |= (uint32_t)in << k;
        }
        uint32_t pnib = inf & leaf;                       // in-frustum leaves pass
        const uint32_t need = inf & ~leaf;                // in-frustum internal nodes
        if (need) {
            const float* c = t.cov;
            const size_t np = t.n_pad;
            float4 cv[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) cv[q] = __ldg(reinterpret_cast<const float4*>(c + q * np) + i);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!((need >> k) & 1u)) continue;
                float s6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    s6[q] = k == 0 ? cv[q].x : k == 1 ? cv[q].y : k == 2 ? cv[q].z : cv[q].w;
                float a, b, cc, lam;
                ewa_cov2d(cam, vz[k], txtz[k], tytz[k], s6, a, b, cc, lam);
                const float R2d = fm(3.0f, fsq(lam));
                if (R2d <= cam.tau_R) pnib |= 1u << k;
            }
        }
        // assemble 32-bit words: lanes 8j..8j+7 hold the nibbles of word j
        uint32_t w = pnib << ((lane & 7) << 2);
        w |= __shfl_xor_sync(0xffffffffu, w, 1);
        w |= __shfl_xor_sync(0xffffffffu, w, 2);
        w |= __shfl_xor_sync(0xffffffffu, w, 4);
        if ((lane & 7) == 0) pbits[i >> 3] = w;
    }
}

void launch_filter_pred(const DevTree& t, const DevCamera& cam, uint32_t* pbits, int blocks,
                        cudaStream_t s)
{
    const uint32_t n_chunks = t.n_pad >> 2;
    int need = (int)((n_chunks + 255) / 256);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    filter_pred_kernel<<<blocks, 256, 0, s>>>(t, cam, pbits);
}

// ---------------------------------------------------------------------------
// Ancestor filter + compaction (persistent, dynamic tiles, decoupled look-back)
// ---------------------------------------------------------------------------

// Ancestor filter of one node with P: does any node of AP(n) (parent first) pass
// R&L?  The path is read in batches of 8 independent loads, then the 8 P bits
// are gathered together, so a walk costs ceil(depth / 8) x 2 round trips.
__device__ __forceinline__ bool ancestor_blocked(const DevTree& t, const uint32_t* __restrict__ pbits,
                                                 uint32_t n)
{
    for (uint32_t k0 = 0; k0 < t.depth; k0 += 8) {
        uint32_t a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            a[q] = (k0 + q < t.depth) ? __ldg(t.ap + (size_t)(k0 + q) * t.n_pad + n) : kApPad;
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = a[q] != kApPad ? __ldg(pbits + (a[q] >> 5)) : 0u;
        bool end = false;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (a[q] == kApPad) { end = true; break; }
            if ((w[q] >> (a[q] & 31)) & 1u) return true;
        }
        if (end) return false;
    }
    return false;
}

__global__ void __launch_bounds__(kFilterThreads) filter_anc_compact_kernel(
    DevTree t, const uint32_t* __restrict__ pbits, uint32_t* __restrict__ sel,
    unsigned long long* lookback, FrameState* st)
{
    __shared__ uint32_t s_cnt[kFilterItems * 8];
    __shared__ uint32_t s_warp_tot[4];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_prefix;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_tiles = (t.n + kFilterTile - 1) / kFilterTile;
    const uint32_t tag = st->epoch * 16u + 0u;
    const uint32_t lt_mask = (1u << lane) - 1u;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&st->tickets[kTicketCompact], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= n_tiles) break;
        const uint32_t base = tile * kFilterTile;
        uint32_t pw[kFilterItems];
#pragma unroll
        for (int it = 0; it < kFilterItems; ++it) {
            const uint32_t n = base + it * kFilterThreads + tid;
            pw[it] = n < t.n ? __ldg(pbits + (n >> 5)) : 0u;
        }
        uint32_t ballots[kFilterItems];
#pragma unroll
        for (int it = 0; it < kFilterItems; ++it) {
            const uint32_t n = base + it * kFilterThreads + tid;
            bool keep = n < t.n && ((pw[it] >> (n & 31)) & 1u);
            if (keep) keep = !ancestor_blocked(t, pbits, n);
            ballots[it] = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_cnt[it * 8 + warp] = __popc(ballots[it]);
        }
        __syncthreads();
        // exclusive scan of the 128 (item, warp) counts in id order
        uint32_t v = 0, incl = 0;
        if (tid < kFilterItems * 8) {
            v = s_cnt[tid];
            incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += u;
            }
            if (lane == 31) s_warp_tot[warp] = incl;
        }
        __syncthreads();
        if (tid < kFilterItems * 8) {
            uint32_t off = 0;
            for (uint32_t w = 0; w < warp; ++w) off += s_warp_tot[w];
            s_cnt[tid] = off + incl - v;
        }
        if (warp == 0) {
            const uint32_t total = s_warp_tot[0] + s_warp_tot[1] + s_warp_tot[2] + s_warp_tot[3];
            uint32_t prefix = 0;
            if (tile == 0) {
                if (lane == 0) st_release_u64(lookback + tile, lb_pack(tag, kFlagIncl, total));
            } else {
                if (lane == 0) st_release_u64(lookback + tile, lb_pack(tag, kFlagAgg, total));
                prefix = warp_lookback(lookback, tile, tag, st, 0x100u);
                if (lane == 0) st_release_u64(lookback + tile, lb_pack(tag, kFlagIncl, prefix + total));
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (tile == n_tiles - 1) st->M = prefix + total;
            }
        }
        __syncthreads();
        const uint32_t prefix = s_prefix;
#pragma unroll
        for (int it = 0; it < kFilterItems; ++it) {
            const uint32_t b = ballots[it];
            if ((b >> lane) & 1u) {
                const uint32_t pos = prefix + s_cnt[it * 8 + warp] + __popc(b & lt_mask);
                sel[pos] = base + it * kFilterThreads + tid;
            }
        }
        __syncthreads();
    }
}

void launch_filter_anc_compact(const DevTree& t, const uint32_t* pbits, uint32_t* sel,
                               unsigned long long* lookback, FrameState* st, int blocks,
                               cudaStream_t s)
{
    const int n_tiles = (int)((t.n + kFilterTile - 1) / kFilterTile);
    if (blocks > n_tiles) blocks = n_tiles;
    if (blocks < 1) blocks = 1;
    filter_anc_compact_kernel<<<blocks, kFilterThreads, 0, s>>>(t, pbits, sel, lookback, st);
}

int occ_filter_pred()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, filter_pred_kernel, 256, 0);
    return b > 0 ? b : 1;
}

int occ_filter_anc()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, filter_anc_compact_kernel, kFilterThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
