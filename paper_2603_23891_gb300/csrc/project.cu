// Projection, SH colour, scene-adaptive shrinking and Gaussian-tile key
// emission (§3.1, §3.3) on sm_103a.
//
// Two passes.  project_kernel: one thread per selected Gaussian computes the
// splat record (centre, conic, log-domain skip threshold, opacity, depth,
// colour, footprint radius), its tile rectangle and pair count, each tile of
// 256 Gaussians its pair total, and the histograms of the four depth digits of
// the sort keys (weighted by pair count).  emit_kernel: exclusive prefixes of those
// totals give every Gaussian its first pair slot, so pairs are emitted in
// selection order (the tie-break of the stable (tile | depth) sort).
#include "project_impl.cuh"

namespace fgs {


// Pass 1: one thread per selected Gaussian.  Writes the splat record, a 16-byte
// footprint record {x0, x1, y0, y1 (u16), pair count, depth bits} and, per tile
// of 256 Gaussians, the tile's pair total.  No inter-block dependency.
__global__ void __launch_bounds__(kProjThreads) project_kernel(
    DevTree t, DevCamera cam, const uint32_t* __restrict__ sel, float* __restrict__ splat,
    uint4* __restrict__ foot, uint32_t* __restrict__ tile_total, FrameState* st)
{
    __shared__ uint32_t s_warp_tot[kProjThreads / 32];
    __shared__ uint32_t s_dhist[4][256];      // depth digits, weighted by pair count
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t M = st->M;
    const uint32_t n_tiles = (M + kProjThreads - 1) / kProjThreads;
    for (int i = tid; i < 4 * 256; i += kProjThreads) (&s_dhist[0][0])[i] = 0;
    __syncthreads();

    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t m = tile * kProjThreads + tid;
        uint32_t cnt = 0;
        if (m < M) cnt = proj::project_one(t, cam, __ldg(sel + m), m, splat, foot);
        if (cnt) {
            // every pair of a Gaussian carries its depth: the four depth digits of
            // the (tile | depth) keys are counted here, once per Gaussian
            const uint32_t d = foot[m].w;
#pragma unroll
            for (int p = 0; p < 4; ++p) atomicAdd(&s_dhist[p][(d >> (8 * p)) & 0xFFu], cnt);
        }
        const uint32_t emitting = __popc(__ballot_sync(0xffffffffu, cnt > 0));
        if (lane == 0 && emitting) atomicAdd(&st->n_emitting, emitting);
        const uint32_t wsum = warp_sum_u32(cnt);
        if (lane == 0) s_warp_tot[warp] = wsum;
        __syncthreads();
        if (tid == 0) {
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kProjThreads / 32; ++w) tot += s_warp_tot[w];
            tile_total[tile] = tot;
        }
        __syncthreads();
    }
    for (int i = tid; i < 4 * 256; i += kProjThreads) {
        const uint32_t c = (&s_dhist[0][0])[i];
        if (c) atomicAdd(&st->hist[0][0] + i, c);
    }
}

// Pass 2: pair slots and key emission.  Block b takes kEmitTiles consecutive
// Gaussian tiles; its first slot is the sum of all earlier tile totals (a block
// reduction, no waiting on other blocks).  Within a tile a block scan orders
// the Gaussians, and each warp writes its pairs with consecutive lanes on
// consecutive slots.  The radix digit histograms of the tile digits are
// accumulated here, per block in shared memory (the depth digits, equal for
// all pairs of a Gaussian, were counted by the projection).
__global__ void __launch_bounds__(kProjThreads) emit_kernel(
    DevCamera cam, const uint4* __restrict__ foot, const uint32_t* __restrict__ tile_total,
    unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals, unsigned long long cap,
    FrameState* st)
{
    __shared__ uint32_t s_warp_tot[kProjThreads / 32];
    __shared__ unsigned long long s_red[kProjThreads / 32];
    __shared__ uint32_t s_hist[kMaxSortPasses][256];
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int passes = cam.sort_passes;
    for (int i = tid; i < kMaxSortPasses * 256; i += kProjThreads) (&s_hist[0][0])[i] = 0;
    const uint32_t M = st->M;
    const uint32_t n_tiles = (M + kProjThreads - 1) / kProjThreads;
    const uint32_t n_groups = (n_tiles + kEmitTiles - 1) / kEmitTiles;
    bool any = false;
    for (uint32_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        any = true;
        const uint32_t t0 = g * kEmitTiles;
        // exclusive prefix of the group: sum of all earlier tile totals
        unsigned long long part = 0;
        for (uint32_t i = tid; i < t0; i += kProjThreads) part += __ldg(tile_total + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_red[warp] = part;
        __syncthreads();
        unsigned long long prefix = 0;
#pragma unroll
        for (int w = 0; w < kProjThreads / 32; ++w) prefix += s_red[w];
        for (uint32_t tile = t0; tile < t0 + kEmitTiles && tile < n_tiles; ++tile) {
            const uint32_t m = tile * kProjThreads + tid;
            uint4 f = make_uint4(0, 0, 0, 0);
            if (m < M) f = __ldg(foot + m);
            const uint32_t cnt = f.z;
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t up = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += up;
            }
            if (lane == 31) s_warp_tot[warp] = incl;
            __syncthreads();
            uint32_t off = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kProjThreads / 32; ++w) {
                const uint32_t tw = s_warp_tot[w];
                off += (w < (int)warp) ? tw : 0u;
                total += tw;
            }
            const unsigned long long wfirst = prefix + off;
            const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - cnt;
            const int32_t x0 = (int32_t)(f.x & 0xFFFFu), x1 = (int32_t)(f.x >> 16);
            const int32_t y0 = (int32_t)(f.y & 0xFFFFu);
            const int32_t rw = x1 - x0;
            if (lane == 0 && wtot && wfirst + wtot > cap) set_status(st, kErrCapacity, 0x300u);
            for (uint32_t q0 = 0; q0 < wtot; q0 += 32) {
                const uint32_t q = q0 + lane;
                // owner of pair q: smallest lane whose inclusive count exceeds q
                uint32_t lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t probe = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                    if (probe <= q) lo += step;
                }
                const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, lo);
                const int32_t o_x0 = __shfl_sync(0xffffffffu, x0, lo);
                const int32_t o_rw = __shfl_sync(0xffffffffu, rw, lo);
                const int32_t o_y0 = __shfl_sync(0xffffffffu, y0, lo);
                const uint32_t o_d = __shfl_sync(0xffffffffu, f.w, lo);
                const uint32_t o_m = __shfl_sync(0xffffffffu, m, lo);
                if (q < wtot) {
                    const unsigned long long idx = wfirst + q;
                    if (idx < cap) {
                        const int32_t k = (int32_t)(q - o_excl);
                        const int32_t ty = o_y0 + k / o_rw;
                        const int32_t tx = o_x0 + k % o_rw;
                        const unsigned long long tl = (unsigned long long)(ty * cam.tiles_x + tx);
                        const unsigned long long key = (tl << 32) | o_d;
                        keys[idx] = key;
                        vals[idx] = o_m;
                        for (int p = 4; p < passes; ++p)     // tile digits (depth: projection)
                            atomicAdd(&s_hist[p][(uint32_t)(key >> (8 * p)) & 0xFFu], 1u);
                    }
                }
            }
            prefix += total;
            if (tile == n_tiles - 1 && tid == 0) st->n_pairs = prefix;
            __syncthreads();
        }
    }
    if (!any) return;
    __syncthreads();
    for (int i = 4 * 256 + tid; i < passes * 256; i += kProjThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&st->hist[0][0] + i, c);
    }
}

void launch_project_emit(const DevTree& t, const DevCamera& cam, const uint32_t* sel,
                         float* splat, uint4* foot, uint32_t* tile_total,
                         unsigned long long* keys, uint32_t* vals, unsigned long long cap,
                         FrameState* st, int proj_blocks, int emit_blocks, cudaStream_t s)
{
    if (proj_blocks < 1) proj_blocks = 1;
    if (emit_blocks < 1) emit_blocks = 1;
    launch_pdl(project_kernel, proj_blocks, kProjThreads, 0, s, t, cam, sel, splat, foot, tile_total,
               st);
    launch_pdl(emit_kernel, emit_blocks, kProjThreads, 0, s, cam, (const uint4*)foot,
               (const uint32_t*)tile_total, keys, vals, cap, st);
}

int occ_project()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, project_kernel, kProjThreads, 0);
    return b > 0 ? b : 1;
}

int occ_emit()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, emit_kernel, kProjThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
