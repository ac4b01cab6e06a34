// Onesweep LSD radix sort of the Gaussian-tile pairs by (tile | depth) key,
// and per-tile ranges of the sorted list (sm_103a).
//
// Design after Adinets & Merrill, "Onesweep: A Faster Least Significant Digit
// Radix Sort for GPUs" (2022): the digit histograms of every 8-bit digit are
// known up front (accumulated while the keys are emitted), then each digit
// pass is a single sweep in which a
// block ranks its tile of 4096 keys locally (warp match + per-warp counters,
// stable), publishes its per-digit counts, looks back over preceding tiles for
// their counts (decoupled look-back, bounded spins) and scatters through
// shared memory so that each digit run is written contiguously.  Stability
// keeps emission order among equal keys, i.e. the selection rank.
#include "fgs_internal.cuh"

namespace fgs {

struct SortSmem {
    uint32_t whist[kSortThreads / 32][256];   // per-warp digit counters, then warp offsets
    uint32_t lbase[256];                      // tile-local start of each digit
    uint32_t gbase[256];                      // global start of each digit for this tile
    uint32_t goff[256];                       // global digit offsets (exclusive scan of hist)
    uint32_t scan_tmp[kSortThreads / 32];
    uint32_t tile;
    uint32_t pad_[3];
    unsigned long long keys[kSortTile];
    uint32_t vals[kSortTile];
};

__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* tmp, uint32_t& total)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    uint32_t off = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t t = tmp[w];
        off += (w < (int)warp) ? t : 0u;
        total += t;
    }
    __syncthreads();
    return off + incl - v;
}

__global__ void __launch_bounds__(kSortThreads, 2) sort_pass_kernel(
    const unsigned long long* __restrict__ in_k, const uint32_t* __restrict__ in_v,
    unsigned long long* __restrict__ out_k, uint32_t* __restrict__ out_v, unsigned long long cap,
    int pass, unsigned long long* lookback, FrameState* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& S = *reinterpret_cast<SortSmem*>(smem_raw);
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t shift = 8u * (uint32_t)pass;
    unsigned long long nll = st->n_pairs;
    nll = nll < cap ? nll : cap;
    const uint32_t n = (uint32_t)nll;
    const uint32_t n_tiles = (n + kSortTile - 1) / kSortTile;
    const uint32_t tag = st->epoch * 16u + 2u + (uint32_t)pass;
    const uint32_t lt_mask = (1u << lane) - 1u;

    {
        uint32_t total;
        const uint32_t h = st->hist[pass][tid];
        S.goff[tid] = block_excl_scan_256(h, S.scan_tmp, total);
    }

    // Block b takes tile b first, then tickets hand out tiles gridDim.x, ... in
    // order (one atomic round trip fewer on the critical path).  The grid is
    // the resident capacity, so every earlier tile's block runs and each
    // look-back wait ends.
    bool first = true;
    for (;;) {
        if (tid == 0)
            S.tile = first ? blockIdx.x : gridDim.x + atomicAdd(&st->tickets[kTicketSortBase + pass], 1u);
        first = false;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) S.whist[w][tid] = 0;
        __syncthreads();
        const uint32_t tile = S.tile;
        if (tile >= n_tiles) break;
        const uint32_t base = tile * kSortTile + warp * (kSortTileItems * 32);

        unsigned long long k[kSortTileItems];
        uint32_t rank[kSortTileItems];
#pragma unroll
        for (int i = 0; i < kSortTileItems; ++i) {
            const uint32_t idx = base + i * 32 + lane;
            k[i] = idx < n ? __ldg(in_k + idx) : ~0ull;
        }
        // stable local ranking: order (warp, item, lane) is the input order.  The
        // lanes holding the same digit are found with one ballot per digit bit.
#pragma unroll
        for (int i = 0; i < kSortTileItems; ++i) {
            const uint32_t idx = base + i * 32 + lane;
            const bool valid = idx < n;
            const uint32_t d = (uint32_t)((k[i] >> shift) & 0xFFu);
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool on = (d >> bit) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, on);
                peers &= on ? bb : ~bb;
            }
            uint32_t b = 0;
            if (valid) b = S.whist[warp][d];
            __syncwarp();
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) S.whist[warp][d] = b + __popc(peers);
            __syncwarp();
            rank[i] = b + __popc(peers & lt_mask);
        }
        __syncthreads();
        // per digit: exclusive prefix across warps, tile count
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t c = S.whist[w][tid];
            S.whist[w][tid] = cnt;
            cnt += c;
        }
        // publish, then look back for the digit's count in all earlier tiles
        unsigned long long* lb = lookback + (size_t)tile * 256 + tid;
        uint32_t prefix = 0;
        if (tile == 0) {
            st_lb_u64(lb, lb_pack(tag, kFlagIncl, cnt));
        } else {
            // each round trip reads this digit's entry of up to 8 preceding tiles at once
            st_lb_u64(lb, lb_pack(tag, kFlagAgg, cnt));
            const uint32_t tg = tag & 0x3FFFFFFFu;
            int j = (int)tile - 1;
            uint64_t spins = 0;
            while (j >= 0) {
                unsigned long long e[kLookbackRows];
#pragma unroll
                for (int q = 0; q < kLookbackRows; ++q)
                    e[q] = (j - q >= 0) ? ld_lb_u64(lookback + (size_t)(j - q) * 256 + tid) : 0ull;
                int used = 0;
                bool done = false;
#pragma unroll
                for (int q = 0; q < kLookbackRows; ++q) {
                    if (j - q < 0) { done = true; break; }
                    const unsigned long long flag = (e[q] >> 32) & 3ull;
                    if ((uint32_t)(e[q] >> 34) != tg || flag == 0) break;
                    prefix += (uint32_t)e[q];
                    ++used;
                    if (flag == kFlagIncl) { done = true; break; }
                }
                if (done) break;
                if (used == 0) {
                    if (++spins > kSpinLimit) { set_status(st, kErrTimeout, 0x400u + (uint32_t)pass); break; }
                    __nanosleep(20);
                }
                j -= used;
            }
            st_lb_u64(lb, lb_pack(tag, kFlagIncl, prefix + cnt));
        }
        uint32_t tile_total;
        const uint32_t lb_start = block_excl_scan_256(cnt, S.scan_tmp, tile_total);
        S.lbase[tid] = lb_start;
        S.gbase[tid] = S.goff[tid] + prefix;
        __syncthreads();
        // stage the tile in shared memory in sorted order
#pragma unroll
        for (int i = 0; i < kSortTileItems; ++i) {
            const uint32_t idx = base + i * 32 + lane;
            if (idx < n) {
                const uint32_t d = (uint32_t)((k[i] >> shift) & 0xFFu);
                const uint32_t pos = S.lbase[d] + S.whist[warp][d] + rank[i];
                S.keys[pos] = k[i];
                S.vals[pos] = __ldg(in_v + idx);    // values are read once, at staging
            }
        }
        __syncthreads();
        // scatter: consecutive positions of one digit go to consecutive addresses
        for (uint32_t j = tid; j < tile_total; j += kSortThreads) {
            const unsigned long long key = S.keys[j];
            const uint32_t d = (uint32_t)((key >> shift) & 0xFFu);
            const uint32_t pos = S.gbase[d] + (j - S.lbase[d]);
            if (pos < n) {          // always true unless a look-back timed out
                out_k[pos] = key;
                out_v[pos] = S.vals[j];
            }
        }
        __syncthreads();
    }
}

int launch_sort(unsigned long long* keys0, uint32_t* vals0, unsigned long long* keys1,
                uint32_t* vals1, unsigned long long cap, int passes,
                unsigned long long* lookback, FrameState* st, int sort_blocks, cudaStream_t s)
{
    cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SortSmem));
    for (int p = 0; p < passes; ++p) {
        const bool even = (p & 1) == 0;
        launch_pdl(sort_pass_kernel, sort_blocks, kSortThreads, sizeof(SortSmem), s,
                   even ? keys0 : keys1, even ? vals0 : vals1, even ? keys1 : keys0,
                   even ? vals1 : vals0, cap, p, lookback, st);
    }
    return passes;
}

size_t sort_smem_bytes() { return sizeof(SortSmem); }

__global__ void tile_ranges_kernel(const unsigned long long* __restrict__ keys,
                                   unsigned long long cap, uint2* __restrict__ ranges,
                                   const FrameState* st)
{
    grid_dep_wait();
    grid_dep_trigger();
    unsigned long long nll = st->n_pairs;
    nll = nll < cap ? nll : cap;
    const uint32_t n = (uint32_t)nll;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t tl = (uint32_t)(__ldg(keys + i) >> 32);
        if (i == 0 || (uint32_t)(__ldg(keys + i - 1) >> 32) != tl) ranges[tl].x = i;
        if (i == n - 1 || (uint32_t)(__ldg(keys + i + 1) >> 32) != tl) ranges[tl].y = i + 1;
    }
}

void launch_tile_ranges(const unsigned long long* keys, unsigned long long cap, uint2* ranges,
                        const FrameState* st, int blocks, cudaStream_t s)
{
    if (blocks < 1) blocks = 1;
    launch_pdl(tile_ranges_kernel, blocks, 256, 0, s, keys, cap, ranges, st);
}

int occ_sort_pass()
{
    cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SortSmem));
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sort_pass_kernel, kSortThreads, sizeof(SortSmem));
    return b > 0 ? b : 1;
}

int occ_tile_ranges()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_ranges_kernel, 256, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
