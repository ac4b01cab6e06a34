// Traversal-free parallel filtering (§3.2) on sm_103a.
//
//  filter_pred        R&L filter: every node independently, P(n) = in-frustum and
//                     (leaf or R_2D = 3 sqrt(lambda_max) <= tau_R).  Streams the
//                     SoA centres with 16-byte loads, skipping each 128-node chunk
//                     whose centres' box lies outside the frustum (none of its
//                     nodes can pass); the covariance is read only for in-frustum
//                     internal nodes (a leaf passes on the frustum test alone).
//                     Output: one bit per node.
//  filter_anc         Ancestor filter: a node with P walks its ancestor path AP
//                     (parent first, stopping at the first ancestor with P); one bit
//                     per node for the survivors, and the survivors of every
//                     compaction tile counted.
//  compact_counted    Stream compaction of the survivor bits into ascending node ids
//                     (each tile's first slot from the counts of the tiles before
//                     it, popcounts, block scan).
//  compact            The same compaction without the counts (decoupled look-back
//                     across tiles): the level-wise filter, the batched form and
//                     the allocation-free entry point.
#include "fgs_internal.cuh"

namespace fgs {

__global__ void frame_begin_kernel(FrameState* st, uint32_t* tile_cnt, int n_tiles, uint32_t* sel_cnt,
                                   int n_sel_tiles)
{
    grid_dep_wait();
    grid_dep_trigger();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        st->epoch = st->epoch + 1;
        st->M = 0;
        st->n_pairs = 0;
        st->blend_entries = 0;
        st->blend_evals = 0;
        st->blend_hits = 0;
        st->blend_active = 0;
        st->n_emitting = 0;
        st->filter_in_frustum = 0;
        st->filter_cov_nodes = 0;
        st->filter_chunks = 0;
    }
    if (tid < 16) st->tickets[tid] = 0;
    for (int i = tid; i < n_tiles; i += gridDim.x * blockDim.x) tile_cnt[i] = 0;
    for (int i = tid; i < n_sel_tiles; i += gridDim.x * blockDim.x) sel_cnt[i] = 0;
}

void launch_frame_begin(FrameState* st, uint32_t* tile_cnt, int n_tiles, uint32_t* sel_cnt, int n_sel_tiles,
                        cudaStream_t s)
{
    int blocks = (n_tiles + 255) / 256;
    blocks = blocks < 8 ? 8 : blocks;
    launch_pdl(frame_begin_kernel, blocks, 256, 0, s, st, tile_cnt, n_tiles, sel_cnt, n_sel_tiles);
}

// ---------------------------------------------------------------------------
// R&L predicate: 4 consecutive nodes per thread, bits assembled per warp.
// count_st (counting frames only, else null): in-frustum nodes, in-frustum
// internal nodes and the chunks read are added to its filter counters, one
// atomic per warp.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) filter_pred_kernel(DevTree t, DevCamera cam, uint32_t* pbits,
                                                          FrameState* count_st)
{
    __shared__ FrustumPlanes s_planes;
    if (threadIdx.x == 0) frustum_planes(cam, s_planes);
    __syncthreads();
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_box = t.n_pad >> 7;                  // 128-node chunks
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t n_in = 0, n_cov = 0, n_read = 0;
    // warp g takes chunks g, g + W, g + 2W, ... (W warps), 32 at a time: lane l tests
    // the box of the l-th; a chunk whose box lies outside the frustum has no node with
    // P, so its centres are not read and its P bits are written as 0; the others are
    // read by the whole warp, 4 nodes a lane, the next one prefetched into L2
    for (uint32_t cb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cb < n_box; cb += 32u * n_warps) {
        const uint32_t cl = cb + lane * n_warps;
        bool out = true;
        if (cl < n_box) {
            out = chunk_outside(s_planes, __ldg(t.cbox + 2 * cl), __ldg(t.cbox + 2 * cl + 1));
            if (out) reinterpret_cast<uint4*>(pbits)[cl] = make_uint4(0u, 0u, 0u, 0u);
        }
        uint32_t todo = __ballot_sync(0xffffffffu, !out);
        while (todo) {
            const uint32_t j = (uint32_t)__ffs(todo) - 1u;
            todo &= todo - 1u;
            if (todo) {
                const uint32_t cn = cb + ((uint32_t)__ffs(todo) - 1u) * n_warps;
                const float* nx = t.mu + ((size_t)cn << 7) + (lane << 2);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nx));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + t.n_pad));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + 2 * (size_t)t.n_pad));
            }
            const uint32_t i = ((cb + j * n_warps) << 5) + lane;   // this lane's 4 nodes
            const uint32_t n0 = i << 2;
            ++n_read;
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
            n_in += __popc(inf);
            n_cov += __popc(need);
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
    if (count_st) {
        const uint32_t a = warp_sum_u32(n_in), b = warp_sum_u32(n_cov);
        if (lane == 0) {
            atomicAdd(&count_st->filter_in_frustum, (unsigned long long)a);
            atomicAdd(&count_st->filter_cov_nodes, (unsigned long long)b);
            atomicAdd(&count_st->filter_chunks, (unsigned long long)n_read);
        }
    }
}

// The box of the centres of each 128 consecutive nodes (one warp a chunk, four
// nodes a lane); a chunk of padding only gets lo.x > hi.x.  Run after every change
// of the centres (tree upload, parameter map).
__global__ void __launch_bounds__(256) chunk_boxes_kernel(DevTree t)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_box = t.n_pad >> 7;
    float4* box = const_cast<float4*>(t.cbox);
    for (uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < n_box;
         b += (gridDim.x * blockDim.x) >> 5) {
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t n = (b << 7) + (lane << 2) + k;
            if (n < t.n)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float v = t.mu[(size_t)q * t.n_pad + n];
                    lo[q] = fminf(lo[q], v);
                    hi[q] = fmaxf(hi[q], v);
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
                hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
            }
        if (lane == 0) {
            box[2 * b] = make_float4(lo[0], lo[1], lo[2], 0.0f);
            box[2 * b + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
        }
    }
}

void launch_chunk_boxes(const DevTree& t, int sms, cudaStream_t s)
{
    const uint32_t n_box = t.n_pad >> 7;
    int blocks = (int)((n_box + 7) / 8);
    if (blocks > sms * 8) blocks = sms * 8;
    if (blocks < 1) blocks = 1;
    chunk_boxes_kernel<<<blocks, 256, 0, s>>>(t);
}

void launch_filter_pred(const DevTree& t, const DevCamera& cam, uint32_t* pbits, FrameState* count_st,
                        int blocks, cudaStream_t s)
{
    const uint32_t n_chunks = t.n_pad >> 2;
    int need = (int)((n_chunks + 255) / 256);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    launch_pdl(filter_pred_kernel, blocks, 256, 0, s, t, cam, pbits, count_st);
}

// ---------------------------------------------------------------------------
// Ancestor filter + compaction (persistent, dynamic tiles, decoupled look-back)
// ---------------------------------------------------------------------------

// Ancestor filter (§3.2): sel(n) = P(n) and no node of AP(n) has P.  One node per
// lane, a warp per 32-node word of the bit arrays; warp g takes words g, g + W,
// g + 2W, ... (W warps in the grid), so the words of the frustum's id ranges spread
// over every warp.  Lane i loads the P bits of the warp's i-th next word, so one
// load brings 32 words' bits and a word without a P bit costs a ballot.  A node
// with P reads up to 16 levels of its ancestor path in one batch of independent
// loads, then the ancestors' P bits, so a walk costs two dependent round trips
// for trees up to 16 levels deep.  The P bits of the lowest kAncCacheWords * 32
// node ids sit in shared memory: with level-major ids those are the upper levels
// every path crosses.  (Walking two words at a time, with their loads in flight
// together, measured no faster: fewer warps fit.)
__device__ __forceinline__ bool ancestor_blocked16(const DevTree& t, const uint32_t* __restrict__ pbits,
                                                   const uint32_t* s_pb, uint32_t cached_words,
                                                   uint32_t n)
{
    for (uint32_t k0 = 0; k0 < t.depth; k0 += 16) {
        uint32_t a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            a[q] = (k0 + q < t.depth) ? __ldg(t.ap + (size_t)(k0 + q) * t.n_pad + n) : kApPad;
        uint32_t w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint32_t wi = a[q] >> 5;
            w[q] = a[q] == kApPad ? 0u : (wi < cached_words ? s_pb[wi] : __ldg(pbits + wi));
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (a[q] == kApPad) return false;
            if ((w[q] >> (a[q] & 31)) & 1u) return true;
        }
    }
    return false;
}

__global__ void __launch_bounds__(256) filter_anc_kernel(DevTree t, const uint32_t* __restrict__ pbits,
                                                         uint32_t* __restrict__ selbits,
                                                         uint32_t* __restrict__ sel_cnt)
{
    __shared__ uint32_t s_pb[kAncCacheWords];
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_words = t.n_pad >> 5;
    const uint32_t cw = n_words < (uint32_t)kAncCacheWords ? n_words : (uint32_t)kAncCacheWords;
    for (uint32_t i = threadIdx.x; i < cw; i += blockDim.x) s_pb[i] = __ldg(pbits + i);
    __syncthreads();
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wb < n_words; wb += 32u * n_warps) {
        // this lane's word of the warp's next 32 (word indices stay below 2^32:
        // n_words <= 2^26 and 32 W is below 2^21)
        const uint32_t wl = wb + lane * n_warps;
        const uint32_t pw_l = wl < n_words ? __ldg(pbits + wl) : 0u;
        uint32_t act = __ballot_sync(0xffffffffu, pw_l != 0u);
        uint32_t res = 0;
        while (act) {
            const uint32_t i = (uint32_t)__ffs(act) - 1u;
            act &= act - 1u;
            const uint32_t pw = __shfl_sync(0xffffffffu, pw_l, i);
            const uint32_t w = wb + i * n_warps;
            const uint32_t n = (w << 5) + lane;
            bool keep = ((pw >> lane) & 1u) && n < t.n;
            if (keep) keep = !ancestor_blocked16(t, pbits, s_pb, cw, n);
            const uint32_t b = __ballot_sync(0xffffffffu, keep);
            if (lane == i) res = b;
            if (lane == 0 && b) atomicAdd(sel_cnt + w / kSelTileWords, (uint32_t)__popc(b));
        }
        if (wl < n_words) selbits[wl] = res;
    }
}

void launch_filter_anc(const DevTree& t, const uint32_t* pbits, uint32_t* selbits, uint32_t* sel_cnt,
                       int blocks, cudaStream_t s)
{
    const uint32_t n_words = t.n_pad >> 5;
    int need = (int)((n_words * 32 + 255) / 256);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    launch_pdl(filter_anc_kernel, blocks, 256, 0, s, t, pbits, selbits, sel_cnt);
}

// Stream compaction of the selection bits into ascending node ids.  Tiles of
// kCompactWords 32-bit words (4 per thread); popcounts, a block scan, and a
// warp-parallel decoupled look-back across tiles give each word its first slot.
__global__ void __launch_bounds__(256) compact_kernel(const uint32_t* __restrict__ selbits,
                                                      uint32_t n_words, uint32_t* __restrict__ sel,
                                                      uint32_t cap, unsigned long long* lookback,
                                                      FrameState* st)
{
    __shared__ uint32_t s_warp_tot[8];
    __shared__ uint32_t s_tile, s_prefix;
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_tiles = (n_words + kCompactWords - 1) / kCompactWords;
    const uint32_t tag = st->epoch * 16u + 0u;
    // block b takes tile b first, later tiles come from the ticket counter in
    // order (the grid is at most the resident capacity: every look-back wait ends)
    bool first = true;
    for (;;) {
        if (tid == 0) s_tile = first ? blockIdx.x : gridDim.x + atomicAdd(&st->tickets[kTicketCompact], 1u);
        first = false;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= n_tiles) break;
        const uint32_t wbase = tile * kCompactWords + tid * 4;
        uint4 wv = make_uint4(0, 0, 0, 0);
        if (wbase + 3 < n_words) {
            wv = __ldg(reinterpret_cast<const uint4*>(selbits + wbase));
        } else {
            if (wbase < n_words) wv.x = __ldg(selbits + wbase);
            if (wbase + 1 < n_words) wv.y = __ldg(selbits + wbase + 1);
            if (wbase + 2 < n_words) wv.z = __ldg(selbits + wbase + 2);
        }
        const uint32_t c0 = __popc(wv.x), c1 = __popc(wv.y), c2 = __popc(wv.z), c3 = __popc(wv.w);
        const uint32_t cnt = c0 + c1 + c2 + c3;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        if (lane == 31) s_warp_tot[warp] = incl;
        __syncthreads();
        uint32_t off = 0, total = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t tw = s_warp_tot[w];
            off += (w < (int)warp) ? tw : 0u;
            total += tw;
        }
        if (warp == 0) {
            uint32_t prefix = 0;
            if (tile == 0) {
                if (lane == 0) st_lb_u64(lookback + tile, lb_pack(tag, kFlagIncl, total));
            } else {
                if (lane == 0) st_lb_u64(lookback + tile, lb_pack(tag, kFlagAgg, total));
                prefix = warp_lookback(lookback, tile, tag, st, 0x100u);
                if (lane == 0) st_lb_u64(lookback + tile, lb_pack(tag, kFlagIncl, prefix + total));
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (tile == n_tiles - 1) {
                    // more survivors than slots: latch the error, keep M within the buffer
                    const uint32_t m_all = prefix + total;
                    if (m_all > cap) set_status(st, kErrCapacity, 0x110u);
                    st->M = m_all < cap ? m_all : cap;
                }
            }
        }
        __syncthreads();
        // warp-cooperative expansion: the warp's 128 words in order, one bit per lane
        const uint32_t p0 = s_prefix + off + incl - cnt;       // first slot of this lane's words
        const uint32_t lt = (1u << lane) - 1u;
        const uint32_t wbase_warp = tile * kCompactWords + warp * 128;
        for (uint32_t q = 0; q < 128; ++q) {
            const uint32_t owner = q >> 2, sub = q & 3;
            const uint32_t mine = sub == 0 ? wv.x : sub == 1 ? wv.y : sub == 2 ? wv.z : wv.w;
            const uint32_t before = sub == 0 ? 0u : sub == 1 ? c0 : sub == 2 ? c0 + c1 : c0 + c1 + c2;
            const uint32_t wq = __shfl_sync(0xffffffffu, mine, owner);
            if (wq == 0u) continue;
            const uint32_t bq = __shfl_sync(0xffffffffu, p0 + before, owner);
            const uint32_t pos = bq + __popc(wq & lt);
            if (((wq >> lane) & 1u) && pos < cap) sel[pos] = ((wbase_warp + q) << 5) + lane;
        }
        __syncthreads();
    }
}

// Compaction of the frame's selection bits when the Ancestor filter has also
// counted the selected nodes of every kSelTileWords-word tile (sel_cnt): one
// block per tile, one word per thread, takes the tile's first slot as the sum
// of the counts of the tiles before it, so no block waits on another (no
// look-back chain); then popcounts, a block scan and a warp-cooperative bit
// expansion of each warp's 32 words (coalesced stores of ascending ids).
__global__ void __launch_bounds__(kSelTileWords) compact_counted_kernel(const uint32_t* __restrict__ selbits,
                                                                        uint32_t n_words,
                                                                        uint32_t* __restrict__ sel, uint32_t cap,
                                                                        const uint32_t* __restrict__ sel_cnt,
                                                                        FrameState* st)
{
    constexpr int kWarps = kSelTileWords / 32;
    __shared__ uint32_t s_warp_tot[kWarps];
    __shared__ uint32_t s_prefix;
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tile = blockIdx.x;
    const uint32_t n_tiles = (n_words + kSelTileWords - 1) / kSelTileWords;
    const uint32_t w = tile * kSelTileWords + tid;
    const uint32_t wv = w < n_words ? selbits[w] : 0u;       // issued before the prefix loads
    uint32_t part = 0;
    for (uint32_t j = tid; j < tile; j += kSelTileWords) part += sel_cnt[j];
    part = warp_sum_u32(part);
    if (lane == 0) s_warp_tot[warp] = part;
    __syncthreads();
    if (tid == 0) {
        uint32_t p = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) p += s_warp_tot[k];
        s_prefix = p;
    }
    __syncthreads();
    const uint32_t prefix = s_prefix;
    const uint32_t cnt = __popc(wv);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    __syncthreads();                               // s_warp_tot reused
    if (lane == 31) s_warp_tot[warp] = incl;
    __syncthreads();
    uint32_t off = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
        const uint32_t tw = s_warp_tot[k];
        off += (k < (int)warp) ? tw : 0u;
        total += tw;
    }
    if (tid == 0 && tile == n_tiles - 1) {
        // more survivors than slots: latch the error, keep M within the buffer
        const uint32_t m_all = prefix + total;
        if (m_all > cap) set_status(st, kErrCapacity, 0x120u);
        st->M = m_all < cap ? m_all : cap;
    }
    // warp-cooperative expansion: the warp's 32 words in order, one bit per lane
    const uint32_t p0 = prefix + off + incl - cnt;        // first slot of this lane's word
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t wbase_warp = tile * kSelTileWords + warp * 32;
    uint32_t any = __ballot_sync(0xffffffffu, wv != 0u);
    while (any) {
        const uint32_t q = (uint32_t)__ffs(any) - 1u;
        any &= any - 1u;
        const uint32_t wq = __shfl_sync(0xffffffffu, wv, q);
        const uint32_t bq = __shfl_sync(0xffffffffu, p0, q);
        const uint32_t pos = bq + __popc(wq & lt);
        if (((wq >> lane) & 1u) && pos < cap) sel[pos] = ((wbase_warp + q) << 5) + lane;
    }
}

void launch_compact_counted(const uint32_t* selbits, uint32_t n_words, uint32_t* sel, uint32_t cap,
                            const uint32_t* sel_cnt, FrameState* st, cudaStream_t s)
{
    const int n_tiles = (int)((n_words + kSelTileWords - 1) / kSelTileWords);
    launch_pdl(compact_counted_kernel, n_tiles < 1 ? 1 : n_tiles, kSelTileWords, 0, s, selbits, n_words, sel,
               cap, sel_cnt, st);
}

// One warp looks back from tile 1 at tile 0 with a tag whose low four bits
// (15) no frame uses (frames tag epoch * 16 + 0, 2..10), so entry 0 never reads
// as ready and the wait ends by its bound.
__global__ void wait_probe_kernel(const unsigned long long* lb, FrameState* st)
{
    (void)warp_lookback<kProbeSpins>(lb, 1u, 0x3FFFFFFFu, st, kProbeSite);
}

void launch_wait_probe(const unsigned long long* lb, FrameState* st, cudaStream_t s)
{
    wait_probe_kernel<<<1, 32, 0, s>>>(lb, st);
}

void launch_compact(const uint32_t* selbits, uint32_t n_words, uint32_t* sel, uint32_t cap,
                    unsigned long long* lookback, FrameState* st, int blocks, cudaStream_t s)
{
    const int n_tiles = (int)((n_words + kCompactWords - 1) / kCompactWords);
    if (blocks > n_tiles) blocks = n_tiles;
    if (blocks < 1) blocks = 1;
    launch_pdl(compact_kernel, blocks, 256, 0, s, selbits, n_words, sel, cap, lookback, st);
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, filter_anc_kernel, 256, 0);
    return b > 0 ? b : 1;
}

int occ_compact()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, compact_kernel, 256, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
