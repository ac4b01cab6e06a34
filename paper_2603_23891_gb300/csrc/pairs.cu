// Gaussian-tile pairs in (tile, depth, rank) order, sm_103a: tile ranges,
// key scatter and per-tile sort.
//
// The pair list (§3.3: one key-value pair per Gaussian and touched tile, sorted
// before blending) is ordered by tile, then by the Gaussian's depth, then by
// its selection rank.  Instead of a radix sort over the whole (tile | depth)
// key, the pairs are bucketed by tile and each tile's bucket is sorted on its
// own:
//  * the projection counts every pair into its tile (pairs_impl.cuh);
//  * tile_scan_kernel: turns the counts into tile ranges [first, last) and
//    scatter cursors (exclusive prefix, decoupled look-back across scan tiles
//    of 2048 tiles), N_P, and the list of tiles with more than kSegSmall pairs;
//  * scatter_kernel: every pair is written into its tile's bucket at a slot
//    taken from the tile's cursor, as one 64-bit item (depth bits << 32 |
//    rank); the order inside a bucket is arbitrary;
//  * segsort_kernel: each bucket is sorted by item.  (depth, rank) is unique
//    within a tile, so the result does not depend on the scatter order.  Four
//    forms by bucket size: a warp sorts up to 32 items in registers (bitonic
//    network, lanes exchange through shuffles) and up to kSegSmall by depth
//    radix passes through its slice of shared memory (with the fix of
//    equal-depth runs below; a longer run: the network); a block sorts up to
//    kSegSmem items by depth with a stable LSD radix sort in shared memory
//    (and, if two depths are equal, with the bitonic network by (depth, rank)
//    instead); a block sorts a larger bucket with an LSD radix sort over every
//    byte in which the items differ, in chunks, between the bucket and the
//    tile's slots of the key output.  The sorted bucket is written as keys
//    (tile << 32 | depth bits) and values (rank).
#include "pairs_impl.cuh"

namespace fgs {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                 // consecutive tiles per thread (2048 per scan tile)
constexpr int kSegThreads = 256;
constexpr int kScatterRounds = 4;             // enumeration rounds whose cursor increments overlap
constexpr unsigned long long kItemPad = ~0ull;   // sorts after every real item

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m)
{
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b)
{
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a < b ? b : a;
}

// One step (k, j) of the bitonic sorting network on E * 32 items held by a
// warp: item e of lane L is element idx0 + 32 e + L of the sequence (idx0 a
// multiple of 32 E, so a k-block's direction is that of the whole sequence).
// The pair (i, i ^ j) is put in ascending order if i & k is 0, else
// descending.  j >= 32: both items are in the same lane; j < 32: the partner is
// lane L ^ j.
template <int E>
__device__ __forceinline__ void net_step(unsigned long long (&v)[E], uint32_t lane, uint32_t idx0,
                                         uint32_t k, int j)
{
    if (j >= 32) {
        const int je = j >> 5;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & je) == 0) {
                const int e2 = e | je;
                const bool asc = ((idx0 + ((uint32_t)e << 5) + lane) & k) == 0u;
                const unsigned long long a = v[e], b = v[e2];
                const bool sw = asc ? (a > b) : (a < b);
                v[e] = sw ? b : a;
                v[e2] = sw ? a : b;
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const unsigned long long o = shfl_xor_u64(v[e], j);
            const bool asc = ((idx0 + ((uint32_t)e << 5) + lane) & k) == 0u;
            const bool lower = (lane & (uint32_t)j) == 0u;
            v[e] = (lower == asc) ? umin64(v[e], o) : umax64(v[e], o);
        }
    }
}

// Every step with k <= 32 E: sorts the warp's items (ascending if idx0's
// k = 32 E block runs ascending).
template <int E>
__device__ __forceinline__ void net_sort(unsigned long long (&v)[E], uint32_t lane, uint32_t idx0)
{
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) net_step<E>(v, lane, idx0, (uint32_t)k, j);
    }
}

// The steps j = 16 E .. 1 of a larger k, on the warp's items.
template <int E>
__device__ __forceinline__ void net_merge(unsigned long long (&v)[E], uint32_t lane, uint32_t idx0,
                                          uint32_t k)
{
#pragma unroll
    for (int j = 16 * E; j > 0; j >>= 1) net_step<E>(v, lane, idx0, k, j);
}

__device__ __forceinline__ void put_pair(unsigned long long item, uint32_t tile,
                                         unsigned long long* keys_out, uint32_t* vals_out, uint32_t i)
{
    keys_out[i] = ((unsigned long long)tile << 32) | (item >> 32);
    vals_out[i] = (uint32_t)item;
}

// A warp sorts n <= 32 E items of one tile in registers.
template <int E>
__device__ __forceinline__ void warp_sort_bucket(const unsigned long long* items, uint32_t n, uint32_t tile,
                                                 unsigned long long* keys_out, uint32_t* vals_out)
{
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = ((uint32_t)e << 5) + lane;
        v[e] = i < n ? items[i] : kItemPad;
    }
    net_sort<E>(v, lane, 0u);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = ((uint32_t)e << 5) + lane;
        if (i < n) put_pair(v[e], tile, keys_out, vals_out, i);
    }
}

// A block sorts n <= kSegSmem items of one tile by (depth, rank) in shared
// memory s.  The padded sequence of P items (a power of two >= n) is cut into
// chunks of 32 E items, dealt out to the warps: each chunk is sorted in
// registers; then for every larger k the steps j >= 32 E run across the
// sequence (one block barrier each) and the steps j < 32 E chunk by chunk in
// registers.  E = P / 256 up to 8, so every warp holds a chunk.
template <int E>
__device__ void block_bitonic_bucket(unsigned long long* s, const unsigned long long* items, uint32_t n,
                                     uint32_t P, uint32_t tile, unsigned long long* keys_out,
                                     uint32_t* vals_out)
{
    constexpr uint32_t C = 32u * E;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t n_warps = kSegThreads / 32;
    const uint32_t chunks = P / C;
    for (uint32_t c = warp; c < chunks; c += n_warps) {
        unsigned long long v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t i = c * C + ((uint32_t)e << 5) + lane;
            v[e] = i < n ? items[i] : kItemPad;
        }
        net_sort<E>(v, lane, c * C);
#pragma unroll
        for (int e = 0; e < E; ++e) s[c * C + ((uint32_t)e << 5) + lane] = v[e];
    }
    __syncthreads();
    for (uint32_t k = 2 * C; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j >= C; j >>= 1) {
            for (uint32_t i = tid; i < (P >> 1); i += kSegThreads) {
                const uint32_t lo = 2 * i - (i & (j - 1)), hi = lo + j;
                const bool asc = (lo & k) == 0u;
                const unsigned long long a = s[lo], b = s[hi];
                if (asc ? (a > b) : (a < b)) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
            __syncthreads();
        }
        for (uint32_t c = warp; c < chunks; c += n_warps) {
            unsigned long long v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = s[c * C + ((uint32_t)e << 5) + lane];
            net_merge<E>(v, lane, c * C, k);
#pragma unroll
            for (int e = 0; e < E; ++e) s[c * C + ((uint32_t)e << 5) + lane] = v[e];
        }
        __syncthreads();
    }
    // the first n elements of the sorted sequence are the bucket (padding sorts last)
    for (uint32_t i = tid; i < n; i += kSegThreads) put_pair(s[i], tile, keys_out, vals_out, i);
    __syncthreads();
}

__device__ void block_bitonic_any(unsigned long long* s, const unsigned long long* items, uint32_t n,
                                  uint32_t tile, unsigned long long* keys_out, uint32_t* vals_out)
{
    uint32_t P = 512;
    while (P < n) P <<= 1;
    if (P == 512) block_bitonic_bucket<2>(s, items, n, P, tile, keys_out, vals_out);
    else if (P == 1024) block_bitonic_bucket<4>(s, items, n, P, tile, keys_out, vals_out);
    else block_bitonic_bucket<8>(s, items, n, P, tile, keys_out, vals_out);
}

// Scratch of the block radix sorts (shared memory).
struct RadixSmem {
    uint32_t whist[kSegThreads / 32][256];   // per-warp digit counters, then per-warp offsets
    uint32_t dbase[256];                     // next slot of each digit
    uint32_t dcnt[256];                      // a chunk's count of each digit
    uint32_t tmp[kSegThreads / 32];
    unsigned long long vor, vand;            // OR and AND of the bucket's items
};

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* tmp)
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
#pragma unroll
    for (int w = 0; w < kSegThreads / 32; ++w) off += (w < (int)warp) ? tmp[w] : 0u;
    __syncthreads();
    return off + incl - v;
}

// Stable ranking of a chunk of up to 256 I items by 8-bit digit d[it]: item it
// of lane L of warp w is element (w I + it) 32 + L of the chunk, present if
// below nv.  Lanes with the same digit are found with one ballot per digit
// bit.  Afterwards rank[it] is the item's position among its warp's earlier
// items of the same digit, R.whist[w][x] the number of the chunk's items of
// digit x in warps before w, and R.dcnt[x] the chunk's count of digit x.
template <int I>
__device__ __forceinline__ void rank_chunk(const uint32_t (&d)[I], uint32_t nv, RadixSmem& R,
                                           uint32_t (&rank)[I])
{
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int w = 0; w < kSegThreads / 32; ++w) R.whist[w][tid] = 0u;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < I; ++it) {
        const bool valid = (warp * I + it) * 32 + lane < nv;
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
            const bool on = (d[it] >> bit) & 1u;
            const uint32_t bb = __ballot_sync(0xffffffffu, on);
            peers &= on ? bb : ~bb;
        }
        uint32_t b = 0;
        if (valid) b = R.whist[warp][d[it]];
        __syncwarp();
        if (valid && lane == (uint32_t)(__ffs(peers) - 1)) R.whist[warp][d[it]] = b + __popc(peers);
        __syncwarp();
        rank[it] = b + __popc(peers & lt);
    }
    __syncthreads();
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kSegThreads / 32; ++w) {
        const uint32_t c = R.whist[w][tid];
        R.whist[w][tid] = cnt;
        cnt += c;
    }
    R.dcnt[tid] = cnt;
    __syncthreads();
}

// Block-wide OR and AND of 64-bit values (every thread passes its own).
__device__ __forceinline__ void block_or_and(unsigned long long vor, unsigned long long vand, RadixSmem& R)
{
    if (threadIdx.x == 0) {
        R.vor = 0ull;
        R.vand = ~0ull;
    }
    __syncthreads();
    const uint32_t lo_or = __reduce_or_sync(0xffffffffu, (uint32_t)vor);
    const uint32_t hi_or = __reduce_or_sync(0xffffffffu, (uint32_t)(vor >> 32));
    const uint32_t lo_and = __reduce_and_sync(0xffffffffu, (uint32_t)vand);
    const uint32_t hi_and = __reduce_and_sync(0xffffffffu, (uint32_t)(vand >> 32));
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&R.vor, ((unsigned long long)hi_or << 32) | lo_or);
        atomicAnd(&R.vand, ((unsigned long long)hi_and << 32) | lo_and);
    }
    __syncthreads();
}

// Equal depths found after a depth-only sort: the run of equal keys starting at
// i (keys[i - 1] differs, keys[i + 1] is equal) is put in rank order by
// insertion sort of its values, if it is at most kTieRun long; returns false,
// changing nothing, for a longer run.  Only this thread writes the run, and the
// keys (which other threads read) do not change.
constexpr uint32_t kTieRun = 32;
__device__ __forceinline__ bool sort_tie_run(const uint32_t* keys, uint32_t* vals, uint32_t i, uint32_t n)
{
    uint32_t j = i + 1;
    while (j < n && keys[j] == keys[i]) {
        if (j - i >= kTieRun) return false;
        ++j;
    }
    for (uint32_t a = i + 1; a < j; ++a) {
        const uint32_t x = vals[a];
        uint32_t b = a;
        while (b > i && vals[b - 1] > x) {
            vals[b] = vals[b - 1];
            --b;
        }
        vals[b] = x;
    }
    return true;
}

// The same for 64-bit items (depth bits << 32 | rank): a run of equal depths
// sorted by item is sorted by rank.
__device__ __forceinline__ bool sort_tie_run64(unsigned long long* items, uint32_t i, uint32_t n)
{
    const uint32_t d = (uint32_t)(items[i] >> 32);
    uint32_t j = i + 1;
    while (j < n && (uint32_t)(items[j] >> 32) == d) {
        if (j - i >= kTieRun) return false;
        ++j;
    }
    for (uint32_t a = i + 1; a < j; ++a) {
        const unsigned long long x = items[a];
        uint32_t b = a;
        while (b > i && items[b - 1] > x) {
            items[b] = items[b - 1];
            --b;
        }
        items[b] = x;
    }
    return true;
}

// A block sorts n <= 256 I items of one tile by depth with a stable LSD radix
// sort over the depth bytes in which the items differ, items held in registers
// and exchanged through shared memory (skeys / svals) after every pass.  Item i
// of the input order is item it, lane L of warp w with i = (w I + it) 32 + L.
// Equal depths keep that order, which is the scatter's and not the rank order,
// so each run of equal depths is then put in rank order where it lies (by the
// thread holding its first element).  If a run is longer than kTieRun, false is
// returned and nothing is written (the caller sorts the bucket by (depth, rank)
// instead); otherwise the sorted pairs are written and true is returned.
template <int I>
__device__ bool block_radix_bucket(const unsigned long long* items, uint32_t n, uint32_t tile,
                                   unsigned long long* keys_out, uint32_t* vals_out, uint32_t* skeys,
                                   uint32_t* svals, RadixSmem& R)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t key[I], val[I];
    unsigned long long vor = 0ull, vand = ~0ull;
#pragma unroll
    for (int it = 0; it < I; ++it) {
        const uint32_t i = (warp * I + it) * 32 + lane;
        const unsigned long long x = i < n ? items[i] : 0ull;
        key[it] = (uint32_t)(x >> 32);
        val[it] = (uint32_t)x;
        if (i < n) {
            vor |= x;
            vand &= x;
        }
    }
    block_or_and(vor, vand, R);
    const uint32_t diff = (uint32_t)((R.vor & ~R.vand) >> 32);
    for (uint32_t shift = 0; shift < 32; shift += 8) {
        if (((diff >> shift) & 0xFFu) == 0u) continue;
        uint32_t d[I], rank[I];
#pragma unroll
        for (int it = 0; it < I; ++it) d[it] = (key[it] >> shift) & 0xFFu;
        rank_chunk<I>(d, n, R, rank);
        R.dbase[tid] = block_excl_scan(R.dcnt[tid], R.tmp);
        __syncthreads();
#pragma unroll
        for (int it = 0; it < I; ++it) {
            if ((warp * I + it) * 32 + lane < n) {
                const uint32_t pos = R.dbase[d[it]] + R.whist[warp][d[it]] + rank[it];
                skeys[pos] = key[it];
                svals[pos] = val[it];
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < I; ++it) {
            const uint32_t i = (warp * I + it) * 32 + lane;
            if (i < n) {
                key[it] = skeys[i];
                val[it] = svals[i];
            }
        }
        __syncthreads();
    }
    // the depth order into shared memory, then each run of equal depths in rank order
#pragma unroll
    for (int it = 0; it < I; ++it) {
        const uint32_t i = (warp * I + it) * 32 + lane;
        if (i < n) {
            skeys[i] = key[it];
            svals[i] = val[it];
        }
    }
    __syncthreads();
    bool long_run = false;
    for (uint32_t i = tid; i + 1 < n; i += kSegThreads) {
        if (skeys[i + 1] == skeys[i] && (i == 0 || skeys[i - 1] != skeys[i]))
            long_run |= !sort_tie_run(skeys, svals, i, n);
    }
    if (__syncthreads_or(long_run)) return false;
    for (uint32_t i = tid; i < n; i += kSegThreads) {
        keys_out[i] = ((unsigned long long)tile << 32) | skeys[i];
        vals_out[i] = svals[i];
    }
    __syncthreads();
    return true;
}

// A block sorts a bucket of any size by (depth, rank) with stable LSD radix
// passes over bytes of the 64-bit items, each pass a histogram sweep and a
// scatter sweep over chunks of 256 I items, between the bucket (a) and the
// tile's slots of the key output (b) as scratch.  First only the depth bytes in
// which the items differ: equal depths then keep the scatter's order, so each
// run of equal depths is put in rank order where it lies; if a run is longer
// than kTieRun the sort is repeated over every byte in which the items differ
// (rank bytes first, so equal depths end in rank order; the input order does
// not matter, (depth, rank) being unique).  The sorted pairs are written
// to keys_out (which is b) and vals_out.
constexpr int kRadixGlobalItems = 8;
__device__ void radix_global_passes(unsigned long long*& src, unsigned long long*& dst, uint32_t n,
                                    unsigned long long diff, RadixSmem& R)
{
    constexpr int I = kRadixGlobalItems;
    constexpr uint32_t kChunk = 256u * I;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t shift = 0; shift < 64; shift += 8) {
        if (((diff >> shift) & 0xFFull) == 0ull) continue;
        // histogram of the digit over the bucket, then each digit's first slot
        uint32_t total = 0;
        for (uint32_t c0 = 0; c0 < n; c0 += kChunk) {
            const uint32_t nv = n - c0 < kChunk ? n - c0 : kChunk;
            uint32_t d[I], rank[I];
#pragma unroll
            for (int it = 0; it < I; ++it) {
                const uint32_t i = (warp * I + it) * 32 + lane;
                d[it] = i < nv ? (uint32_t)(src[c0 + i] >> shift) & 0xFFu : 0u;
            }
            rank_chunk<I>(d, nv, R, rank);
            total += R.dcnt[tid];
            __syncthreads();
        }
        R.dbase[tid] = block_excl_scan(total, R.tmp);
        __syncthreads();
        // stable scatter, chunk by chunk in order
        for (uint32_t c0 = 0; c0 < n; c0 += kChunk) {
            const uint32_t nv = n - c0 < kChunk ? n - c0 : kChunk;
            unsigned long long x[I];
            uint32_t d[I], rank[I];
#pragma unroll
            for (int it = 0; it < I; ++it) {
                const uint32_t i = (warp * I + it) * 32 + lane;
                x[it] = i < nv ? src[c0 + i] : 0ull;
                d[it] = (uint32_t)(x[it] >> shift) & 0xFFu;
            }
            rank_chunk<I>(d, nv, R, rank);
#pragma unroll
            for (int it = 0; it < I; ++it) {
                if ((warp * I + it) * 32 + lane < nv)
                    dst[R.dbase[d[it]] + R.whist[warp][d[it]] + rank[it]] = x[it];
            }
            __syncthreads();
            R.dbase[tid] += R.dcnt[tid];
            __syncthreads();
        }
        unsigned long long* t = src;
        src = dst;
        dst = t;
    }
}

__device__ void block_radix_global(unsigned long long* a, unsigned long long* b, uint32_t n, uint32_t tile,
                                   unsigned long long* keys_out, uint32_t* vals_out, RadixSmem& R)
{
    const uint32_t tid = threadIdx.x;
    unsigned long long vor = 0ull, vand = ~0ull;
    for (uint32_t i = tid; i < n; i += kSegThreads) {
        const unsigned long long x = a[i];
        vor |= x;
        vand &= x;
    }
    block_or_and(vor, vand, R);
    const unsigned long long diff = R.vor & ~R.vand;
    unsigned long long* src = a;
    unsigned long long* dst = b;
    radix_global_passes(src, dst, n, diff & 0xFFFFFFFF00000000ull, R);
    // each run of equal depths in rank order where it lies; a run longer than
    // kTieRun: the full sort instead
    bool long_run = false;
    for (uint32_t i = tid; i + 1 < n; i += kSegThreads) {
        const uint32_t d = (uint32_t)(src[i] >> 32);
        if ((uint32_t)(src[i + 1] >> 32) == d && (i == 0 || (uint32_t)(src[i - 1] >> 32) != d))
            long_run |= !sort_tie_run64(src, i, n);
    }
    if (__syncthreads_or(long_run)) radix_global_passes(src, dst, n, diff, R);
    // src holds the sorted items; a slot of keys_out (= b) is read and then
    // rewritten by the same thread
    for (uint32_t i = tid; i < n; i += kSegThreads) put_pair(src[i], tile, keys_out, vals_out, i);
    __syncthreads();
}

// A warp sorts n <= 32 I items of one tile by (depth, rank), items in registers
// (item it of lane L is element 32 it + L): stable LSD radix passes over the
// depth bytes in which the items differ, each ranking the digits with one ballot
// per digit bit and the warp's 256 counters (hist), the items exchanged through
// the warp's buffer buf (32 I slots); then each run of equal depths in rank
// order where it lies, and the pairs written.  Returns false, writing nothing,
// if a run is longer than kTieRun (the caller sorts the bucket by the bitonic
// network instead).
template <int I>
__device__ bool warp_radix_small(const unsigned long long* items, uint32_t n, uint32_t tile,
                                 unsigned long long* keys_out, uint32_t* vals_out, unsigned long long* buf,
                                 uint32_t* hist)
{
    const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    unsigned long long x[I];
    uint32_t vor = 0u, vand = ~0u;
#pragma unroll
    for (int it = 0; it < I; ++it) {
        const uint32_t i = ((uint32_t)it << 5) + lane;
        x[it] = i < n ? items[i] : ~0ull;
        if (i < n) {
            vor |= (uint32_t)(x[it] >> 32);
            vand &= (uint32_t)(x[it] >> 32);
        }
    }
    const uint32_t diff = __reduce_or_sync(0xffffffffu, vor) & ~__reduce_and_sync(0xffffffffu, vand);
    for (uint32_t shift = 32; shift < 64; shift += 8) {
        if (((diff >> (shift - 32)) & 0xFFu) == 0u) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) hist[lane * 8 + j] = 0u;
        __syncwarp();
        uint32_t rank[I], dg[I];
#pragma unroll
        for (int it = 0; it < I; ++it) {
            const bool valid = ((uint32_t)it << 5) + lane < n;
            dg[it] = (uint32_t)(x[it] >> shift) & 0xFFu;
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool on = (dg[it] >> bit) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, on);
                peers &= on ? bb : ~bb;
            }
            const uint32_t base = valid ? hist[dg[it]] : 0u;
            __syncwarp();
            if (valid && lane == (uint32_t)(__ffs(peers) - 1)) hist[dg[it]] = base + __popc(peers);
            __syncwarp();
            rank[it] = base + __popc(peers & lt);
        }
        // exclusive scan of the 256 counters, 8 consecutive ones a lane
        uint32_t c[8], sum = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j] = hist[lane * 8 + j];
            sum += c[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        uint32_t run = incl - sum;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hist[lane * 8 + j] = run;
            run += c[j];
        }
        __syncwarp();
#pragma unroll
        for (int it = 0; it < I; ++it)
            if (((uint32_t)it << 5) + lane < n) buf[hist[dg[it]] + rank[it]] = x[it];
        __syncwarp();
#pragma unroll
        for (int it = 0; it < I; ++it) {
            const uint32_t i = ((uint32_t)it << 5) + lane;
            if (i < n) x[it] = buf[i];
        }
        __syncwarp();
    }
#pragma unroll
    for (int it = 0; it < I; ++it) {
        const uint32_t i = ((uint32_t)it << 5) + lane;
        if (i < n) buf[i] = x[it];
    }
    __syncwarp();
    bool long_run = false;
    for (uint32_t i = lane; i + 1 < n; i += 32) {
        const uint32_t d = (uint32_t)(buf[i] >> 32);
        if ((uint32_t)(buf[i + 1] >> 32) == d && (i == 0 || (uint32_t)(buf[i - 1] >> 32) != d))
            long_run |= !sort_tie_run64(buf, i, n);
    }
    if (__any_sync(0xffffffffu, long_run)) return false;
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32) put_pair(buf[i], tile, keys_out, vals_out, i);
    __syncwarp();
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// tile ranges
// ---------------------------------------------------------------------------
// Scan tiles of kScanTile consecutive image tiles, kScanItems a thread; a scan
// tile's first pair slot comes from a decoupled look-back over the totals of
// the scan tiles before it (64-bit look-back entries: epoch tag, flag, 32-bit
// count).  Counts saturate at 2^32 - 1, far above any pair capacity (< 2^31),
// so a saturated prefix still clamps to the capacity and latches the error.
constexpr uint32_t kScanTile = (uint32_t)kScanThreads * kScanItems;
constexpr uint32_t kScanTag = 10u;          // the tile scan's look-back tag, epoch * 16 + 10

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b)
{
    const uint32_t r = a + b;
    return r < a ? 0xFFFFFFFFu : r;
}

// The exclusive prefix of scan tile `tile` over the entries of lb (one full
// warp; lane l reads predecessor base - l, nearest first up to the first
// inclusive entry), with saturating sums; bounded like warp_lookback.
__device__ uint32_t scan_lookback(const unsigned long long* lb, uint32_t tile, uint32_t tag, FrameState* st)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t tg = tag & 0x3FFFFFFFu;
    unsigned long long prefix = 0;
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
        const uint32_t take = inc ? (uint32_t)__ffs(inc) : first_nr;
        unsigned long long v = lane < take ? val : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (prefix > 0xFFFFFFFFull) prefix = 0xFFFFFFFFull;
        if (inc) break;
        if (take == 0) {
            if (++spins > kSpinLimit) {
                set_status(st, kErrTimeout, 0x310u);
                break;
            }
            __nanosleep(20);
        }
        base -= (int)take;
    }
    return (uint32_t)prefix;
}

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(uint32_t* __restrict__ tile_cnt,
                                                                 uint2* __restrict__ ranges,
                                                                 uint32_t n_tiles,
                                                                 uint32_t* __restrict__ large,
                                                                 unsigned long long cap,
                                                                 unsigned long long* lb, FrameState* st)
{
    constexpr int kWarps = kScanThreads / 32;
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_tile, s_prefix;
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_st = (n_tiles + kScanTile - 1) / kScanTile;
    const uint32_t tag = st->epoch * 16u + kScanTag;
    const uint32_t cap32 = (uint32_t)cap;
    // block b takes scan tile b first, later ones come from a ticket counter in
    // order (the grid is at most the resident capacity: every look-back wait ends)
    bool first = true;
    for (;;) {
        if (tid == 0) s_tile = first ? blockIdx.x : gridDim.x + atomicAdd(&st->tickets[kTicketScan], 1u);
        first = false;
        __syncthreads();
        const uint32_t sti = s_tile;
        if (sti >= n_st) break;
        const uint32_t t0 = sti * kScanTile + tid * kScanItems;
        uint32_t c[kScanItems];
        if (t0 + kScanItems <= n_tiles) {
            const uint4 a = *reinterpret_cast<const uint4*>(tile_cnt + t0);
            const uint4 b = *reinterpret_cast<const uint4*>(tile_cnt + t0 + 4);
            c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
            c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < kScanItems; ++i) c[i] = t0 + i < n_tiles ? tile_cnt[t0 + i] : 0u;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) sum = sat_add(sum, c[i]);
        // warp and block scans of the threads' sums (saturating)
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl = sat_add(incl, u);
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t woff = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t tw = s_warp[w];
            if (w < (int)warp) woff = sat_add(woff, tw);
            total = sat_add(total, tw);
        }
        if (warp == 0) {
            uint32_t prefix = 0;
            if (sti == 0) {
                if (lane == 0) st_lb_u64(lb, lb_pack(tag, kFlagIncl, total));
            } else {
                if (lane == 0) st_lb_u64(lb + sti, lb_pack(tag, kFlagAgg, total));
                prefix = scan_lookback(lb, sti, tag, st);
                if (lane == 0) st_lb_u64(lb + sti, lb_pack(tag, kFlagIncl, sat_add(prefix, total)));
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (sti == n_st - 1) {
                    const uint32_t np = sat_add(prefix, total);
                    st->n_pairs = np;
                    if ((unsigned long long)np > cap) set_status(st, kErrCapacity, 0x300u);
                }
            }
        }
        __syncthreads();
        uint32_t off = sat_add(s_prefix, sat_add(woff, incl - (incl == 0xFFFFFFFFu ? 0u : sum)));
        if (incl == 0xFFFFFFFFu) off = 0xFFFFFFFFu;          // saturated: clamps to the capacity below
        // each tile's range [first, last) clamped to the capacity, its scatter cursor,
        // and the list of tiles for the block sort (one reservation per warp and item)
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const uint32_t t = t0 + i;
            const uint32_t a = off < cap32 ? off : cap32;
            const uint32_t end = sat_add(off, c[i]);
            const uint32_t e = end < cap32 ? end : cap32;
            if (t < n_tiles) {
                ranges[t] = make_uint2(a, e);
                tile_cnt[t] = a;
            }
            const bool big = t < n_tiles && e - a > (uint32_t)kSegSmall;
            const uint32_t bm = __ballot_sync(0xffffffffu, big);
            if (bm) {
                uint32_t slot = 0;
                if (lane == 0) slot = atomicAdd(&st->tickets[kTicketLarge], (uint32_t)__popc(bm));
                slot = __shfl_sync(0xffffffffu, slot, 0);
                if (big) large[slot + __popc(bm & ((1u << lane) - 1u))] = t;
            }
            off = end;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// key scatter
// ---------------------------------------------------------------------------
// Every pair of the selected Gaussians m < M (rank m; in the batched form m
// indexes entries view * n_pad + node, and a pair's tile is its view's first
// tile plus the tile in the view) goes to its tile's bucket as
// depth bits << 32 | m.  Slots at or beyond cap are not written (the scan has
// latched FGS_ERR_CAPACITY).  A Gaussian with more than kWarpWidePairs pairs
// is scattered by all lanes of its warp first (scatter_wide).
// One warp's Gaussians (lane L: pair count cnt, footprint f, its view's grid
// width and first tile, rank m) into their tiles' buckets, kScatterRounds rounds
// at a time so that their cursor increments are in flight together; one
// increment per tile and round, the group's lanes taking consecutive slots
// after the returned base.
__device__ __forceinline__ void scatter_warp(uint32_t cnt, const uint4& f, uint32_t tiles_x, uint32_t tbase,
                                             uint32_t m, uint32_t* __restrict__ cursor,
                                             unsigned long long* __restrict__ items, unsigned long long cap)
{
    const uint32_t lane = threadIdx.x & 31;
    const WarpPairs wp(cnt, f.x, f.y, tiles_x, tbase, f.w, m);
    for (uint32_t q0 = 0; q0 < wp.wtot; q0 += 32 * kScatterRounds) {
        uint32_t tile[kScatterRounds], d[kScatterRounds], mm[kScatterRounds], grp[kScatterRounds],
            base[kScatterRounds];
#pragma unroll
        for (int r = 0; r < kScatterRounds; ++r) {
            const bool valid = wp.get(q0 + 32 * r, tile[r], d[r], mm[r]);
            grp[r] = tile_group(valid, tile[r]);
            base[r] = 0;
            if (grp[r] && lane == (uint32_t)(__ffs(grp[r]) - 1))
                base[r] = atomicAdd(cursor + tile[r], (uint32_t)__popc(grp[r]));
        }
#pragma unroll
        for (int r = 0; r < kScatterRounds; ++r) {
            const uint32_t leader = grp[r] ? (uint32_t)(__ffs(grp[r]) - 1) : lane;
            const uint32_t b = __shfl_sync(0xffffffffu, base[r], leader);
            if (grp[r]) {
                const uint32_t pos = b + (uint32_t)__popc(grp[r] & ((1u << lane) - 1u));
                if (pos < cap) items[pos] = ((unsigned long long)d[r] << 32) | mm[r];
            }
        }
    }
}

// The warp's Gaussians with more than kWarpWidePairs pairs (a near, wide
// footprint: up to thousands of tiles), one at a time, by all 32 lanes: one tile
// of the rectangle a lane and step (all distinct tiles, so one cursor increment
// a pair), kWideSlots increments a lane in flight before the items are stored.
constexpr int kWideSlots = 16;
__device__ __forceinline__ void scatter_wide(uint32_t wide, const uint4& f, uint32_t tiles_x, uint32_t tbase,
                                             uint32_t m, uint32_t* __restrict__ cursor,
                                             unsigned long long* __restrict__ items, unsigned long long cap)
{
    const uint32_t lane = threadIdx.x & 31;
    while (wide) {
        const uint32_t b = (uint32_t)__ffs(wide) - 1u;
        wide &= wide - 1u;
        uint4 fb;
        fb.x = __shfl_sync(0xffffffffu, f.x, b);
        fb.y = __shfl_sync(0xffffffffu, f.y, b);
        fb.z = __shfl_sync(0xffffffffu, f.z, b);
        fb.w = __shfl_sync(0xffffffffu, f.w, b);
        const uint32_t mb = __shfl_sync(0xffffffffu, m, b);
        const uint32_t tx = __shfl_sync(0xffffffffu, tiles_x, b), tb = __shfl_sync(0xffffffffu, tbase, b);
        const unsigned long long item = ((unsigned long long)fb.w << 32) | mb;
        for (uint32_t k0 = 0; k0 < fb.z; k0 += 32u * kWideSlots) {
            uint32_t pos[kWideSlots];
#pragma unroll
            for (int r = 0; r < kWideSlots; ++r) {
                const uint32_t k = k0 + (uint32_t)r * 32u + lane;
                pos[r] = k < fb.z ? atomicAdd(cursor + rect_tile(fb, k, tx, tb), 1u) : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int r = 0; r < kWideSlots; ++r)
                if (pos[r] != 0xFFFFFFFFu && pos[r] < cap) items[pos[r]] = item;
        }
    }
}

template <bool kBatch>
__global__ void __launch_bounds__(kProjThreads) scatter_kernel(
    DevCamera cam, const DevCamera* __restrict__ cams, const uint32_t* __restrict__ tile_base,
    uint32_t n_pad, const uint32_t* __restrict__ sel, const uint4* __restrict__ foot,
    uint32_t* __restrict__ cursor, unsigned long long* __restrict__ items, unsigned long long cap,
    FrameState* st)
{
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t M = st->M;
    const uint32_t n_groups = (M + kProjThreads - 1) / kProjThreads;
    for (uint32_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const uint32_t m = g * kProjThreads + threadIdx.x;
        uint4 f = make_uint4(0, 0, 0, 0);
        uint32_t tiles_x = 1, tbase = 0;
        if (m < M) {
            f = __ldg(foot + m);
            if (kBatch) {
                const uint32_t v = __ldg(sel + m) / n_pad;
                tiles_x = (uint32_t)cams[v].tiles_x;
                tbase = __ldg(tile_base + v);
            } else {
                tiles_x = (uint32_t)cam.tiles_x;
            }
        }
        const uint32_t wide = __ballot_sync(0xffffffffu, f.z > kWarpWidePairs);
        if (wide) scatter_wide(wide, f, tiles_x, tbase, m, cursor, items, cap);
        const uint32_t cnt = f.z > kWarpWidePairs ? 0u : f.z;
        if (__ballot_sync(0xffffffffu, cnt != 0) != 0u) scatter_warp(cnt, f, tiles_x, tbase, m, cursor, items, cap);
    }
}

// ---------------------------------------------------------------------------
// per-tile sort
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSegThreads) segsort_kernel(const uint2* __restrict__ ranges,
                                                              uint32_t n_tiles,
                                                              const uint32_t* __restrict__ large,
                                                              unsigned long long* items,
                                                              unsigned long long* keys_out,
                                                              uint32_t* vals_out, FrameState* st)
{
    __shared__ __align__(16) unsigned long long s_items[kSegSmem];
    __shared__ RadixSmem s_radix;
    __shared__ uint32_t s_next;
    grid_dep_wait();
    grid_dep_trigger();
    // large buckets first: one block each; a block's first bucket is its index,
    // later ones come from a ticket counter
    const uint32_t n_large = st->tickets[kTicketLarge];
    bool first = true;
    for (;;) {
        if (threadIdx.x == 0)
            s_next = first ? blockIdx.x : gridDim.x + atomicAdd(&st->tickets[kTicketSegSort], 1u);
        first = false;
        __syncthreads();
        const uint32_t i = s_next;
        __syncthreads();
        if (i >= n_large) break;
        const uint32_t t = large[i];
        const uint2 r = ranges[t];
        const uint32_t n = r.y - r.x;
        unsigned long long* it = items + r.x;
        if (n <= (uint32_t)kSegSmem) {
            uint32_t* sk = reinterpret_cast<uint32_t*>(s_items);
            bool done;
            if (n <= 512u) done = block_radix_bucket<2>(it, n, t, keys_out + r.x, vals_out + r.x, sk, sk + kSegSmem, s_radix);
            else if (n <= 1024u) done = block_radix_bucket<4>(it, n, t, keys_out + r.x, vals_out + r.x, sk, sk + kSegSmem, s_radix);
            else done = block_radix_bucket<8>(it, n, t, keys_out + r.x, vals_out + r.x, sk, sk + kSegSmem, s_radix);
            if (!done) block_bitonic_any(s_items, it, n, t, keys_out + r.x, vals_out + r.x);
        } else {
            block_radix_global(it, keys_out + r.x, n, t, keys_out + r.x, vals_out + r.x, s_radix);
        }
    }
    // small buckets: one warp each, tiles dealt out by warp index; up to 32 items
    // by the bitonic network in registers, more by depth radix passes with the
    // warp's slice of the block sorts' shared memory (free once they are done:
    // the loop above ends on a barrier), the network if a tie run is too long
    const uint32_t gw = (blockIdx.x * kSegThreads + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * kSegThreads) >> 5;
    static_assert(kSegSmem >= kSegThreads / 32 * kSegSmall, "a warp's slice holds a small bucket");
    const uint32_t wl = threadIdx.x >> 5;
    unsigned long long* const wbuf = s_items + wl * kSegSmall;
    uint32_t* const whist = s_radix.whist[wl];
    for (uint32_t t = gw; t < n_tiles; t += nw) {
        const uint2 r = ranges[t];
        const uint32_t n = r.y - r.x;
        if (n == 0u || n > (uint32_t)kSegSmall) continue;
        const unsigned long long* it = items + r.x;
        bool done = true;
        if (n <= 32u) warp_sort_bucket<1>(it, n, t, keys_out + r.x, vals_out + r.x);
        else if (n <= 64u) done = warp_radix_small<2>(it, n, t, keys_out + r.x, vals_out + r.x, wbuf, whist);
        else if (n <= 128u) done = warp_radix_small<4>(it, n, t, keys_out + r.x, vals_out + r.x, wbuf, whist);
        else done = warp_radix_small<8>(it, n, t, keys_out + r.x, vals_out + r.x, wbuf, whist);
        if (!done) {
            if (n <= 64u) warp_sort_bucket<2>(it, n, t, keys_out + r.x, vals_out + r.x);
            else if (n <= 128u) warp_sort_bucket<4>(it, n, t, keys_out + r.x, vals_out + r.x);
            else warp_sort_bucket<8>(it, n, t, keys_out + r.x, vals_out + r.x);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_tile_scan(uint32_t* tile_cnt, uint2* ranges, uint32_t n_tiles, uint32_t* large,
                      unsigned long long cap, unsigned long long* lookback, FrameState* st, int blocks,
                      cudaStream_t s)
{
    const uint32_t n_st = (n_tiles + kScanTile - 1) / kScanTile;
    if (blocks > (int)n_st) blocks = (int)n_st;
    if (blocks < 1) blocks = 1;
    launch_pdl(tile_scan_kernel, blocks, kScanThreads, 0, s, tile_cnt, ranges, n_tiles, large, cap, lookback,
               st);
}

int occ_tile_scan()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_scan_kernel, kScanThreads, 0);
    return b > 0 ? b : 1;
}

void launch_scatter(const DevCamera& cam, const uint4* foot, uint32_t* cursor, unsigned long long* items,
                    unsigned long long cap, FrameState* st, int blocks, cudaStream_t s)
{
    if (blocks < 1) blocks = 1;
    launch_pdl(scatter_kernel<false>, blocks, kProjThreads, 0, s, cam, (const DevCamera*)nullptr,
               (const uint32_t*)nullptr, 0u, (const uint32_t*)nullptr, foot, cursor, items, cap, st);
}

void launch_scatter_batch(const DevCamera* cams, const uint32_t* tile_base, uint32_t n_pad,
                          const uint32_t* sel, const uint4* foot, uint32_t* cursor,
                          unsigned long long* items, unsigned long long cap, FrameState* st, int blocks,
                          cudaStream_t s)
{
    if (blocks < 1) blocks = 1;
    DevCamera none{};
    launch_pdl(scatter_kernel<true>, blocks, kProjThreads, 0, s, none, cams, tile_base, n_pad, sel, foot,
               cursor, items, cap, st);
}

void launch_segsort(const uint2* ranges, uint32_t n_tiles, const uint32_t* large, unsigned long long* items,
                    unsigned long long* keys_out, uint32_t* vals_out, FrameState* st, int blocks,
                    cudaStream_t s)
{
    if (blocks < 1) blocks = 1;
    launch_pdl(segsort_kernel, blocks, kSegThreads, 0, s, ranges, n_tiles, large, items, keys_out, vals_out,
               st);
}

int occ_scatter()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, scatter_kernel<false>, kProjThreads, 0);
    return b > 0 ? b : 1;
}

int occ_segsort()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, segsort_kernel, kSegThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
