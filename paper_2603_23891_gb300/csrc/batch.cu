// Batched multi-view form of the render path (many views of uneven resolution
// per call, sm_103a).
//
// All views go through one sequence of kernels instead of one sequence per view:
//  * bpred_kernel    R&L (§3.2) for every view: each node's centre and covariance
//                    are read once and tested against all V cameras;
//  * banc_kernel     Ancestor filter per view: a node's ancestor path AP is read
//                    once for all views in which the node passed R&L;
//  * compaction      the per-view selection bits are one concatenated bit array
//                    [V][words]; the render path's compaction kernel turns it into
//                    global entries v * n_pad + node (ascending: view, then node);
//  * bproject        projection and shrink of every entry with its view's camera;
//                    pairs are counted into global tile ids (the view's first
//                    tile + the tile), so the render path's tile scan, key
//                    scatter and per-tile sort order every view at once;
//  * bblend over all views' tiles; a CTA finds its view by binary search over
//    the views' first tiles and blends with that camera.
// Per view, selection, pairs, their order and every pixel are those of the
// single-view path with the same camera and tile shape.
#include "blend_impl.cuh"
#include "pairs_impl.cuh"
#include "project_impl.cuh"

namespace fgs {

constexpr int kMaxBatchViews = 64;

__global__ void bframe_begin_kernel(FrameState* st, uint32_t* tile_cnt, uint32_t n_tiles)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        st->epoch = st->epoch + 1;
        st->M = 0;
        st->n_pairs = 0;
    }
    if (tid < 16) st->tickets[tid] = 0;
    for (uint32_t i = tid; i < n_tiles; i += gridDim.x * blockDim.x) tile_cnt[i] = 0;
}

// R&L for V views: 4 consecutive nodes per thread, a warp a 128-node chunk,
// cameras and their frustum planes in shared memory.  Lane v tests the chunk's
// box against view v's frustum: the chunk's centres are read only if some view
// may hold one of them, and evaluated only for those views (a chunk outside a
// view's frustum has no node with P there: its P bits are written as 0); lane l
// tests views l and l + 32.
__global__ void __launch_bounds__(256) bpred_kernel(DevTree t, const DevCamera* __restrict__ cams,
                                                    int V, uint32_t* __restrict__ pbits)
{
    __shared__ DevCamera s_cam[kMaxBatchViews];
    __shared__ FrustumPlanes s_planes[kMaxBatchViews];
    for (int i = threadIdx.x; i < V * (int)(sizeof(DevCamera) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(s_cam)[i] = reinterpret_cast<const uint32_t*>(cams)[i];
    __syncthreads();
    if ((int)threadIdx.x < V) frustum_planes(s_cam[threadIdx.x], s_planes[threadIdx.x]);
    __syncthreads();
    const uint32_t n_chunks = t.n_pad >> 2;
    const uint32_t n_words = t.n_pad >> 5;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;       // a multiple of 32: warps keep 128-node chunks
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_chunks; i += stride) {
        const uint32_t n0 = i << 2;
        const uint32_t c = i >> 5;
        const float4 lo = __ldg(t.cbox + 2 * c), hi = __ldg(t.cbox + 2 * c + 1);
        static_assert(kMaxBatchViews <= 64, "two ballots of views");
        const unsigned long long vmask =
            (unsigned long long)__ballot_sync(0xffffffffu, (int)lane < V && !chunk_outside(s_planes[lane], lo, hi)) |
            ((unsigned long long)__ballot_sync(0xffffffffu, (int)lane + 32 < V &&
                                                                !chunk_outside(s_planes[lane + 32 < kMaxBatchViews ? lane + 32 : 0], lo, hi))
             << 32);
        if (vmask == 0ull) {
            for (int v = 0; v < V; ++v)
                if ((lane & 7) == 0) pbits[(size_t)v * n_words + (i >> 3)] = 0u;
            continue;
        }
        const float4 mx = __ldg(reinterpret_cast<const float4*>(t.mu) + i);
        const float4 my = __ldg(reinterpret_cast<const float4*>(t.mu + t.n_pad) + i);
        const float4 mz = __ldg(reinterpret_cast<const float4*>(t.mu + 2 * (size_t)t.n_pad) + i);
        const uint32_t leaf = (__ldg(t.leaf_bits + (i >> 3)) >> ((i & 7) << 2)) & 0xFu;
        const float xs[4] = {mx.x, mx.y, mx.z, mx.w};
        const float ys[4] = {my.x, my.y, my.z, my.w};
        const float zs[4] = {mz.x, mz.y, mz.z, mz.w};
        float4 cv[6];
        bool have_cov = false;
        for (int v = 0; v < V; ++v) {
            if (!((vmask >> v) & 1ull)) {
                if ((lane & 7) == 0) pbits[(size_t)v * n_words + (i >> 3)] = 0u;
                continue;
            }
            const DevCamera& cam = s_cam[v];
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
            uint32_t pnib = inf & leaf;
            const uint32_t need = inf & ~leaf;
            if (need) {
                if (!have_cov) {
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        cv[q] = __ldg(reinterpret_cast<const float4*>(t.cov + q * (size_t)t.n_pad) + i);
                    have_cov = true;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!((need >> k) & 1u)) continue;
                    float s6[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        s6[q] = k == 0 ? cv[q].x : k == 1 ? cv[q].y : k == 2 ? cv[q].z : cv[q].w;
                    float a, b, cc, lam;
                    ewa_cov2d(cam, vz[k], txtz[k], tytz[k], s6, a, b, cc, lam);
                    if (fm(3.0f, fsq(lam)) <= cam.tau_R) pnib |= 1u << k;
                }
            }
            uint32_t w = pnib << ((lane & 7) << 2);
            w |= __shfl_xor_sync(0xffffffffu, w, 1);
            w |= __shfl_xor_sync(0xffffffffu, w, 2);
            w |= __shfl_xor_sync(0xffffffffu, w, 4);
            if ((lane & 7) == 0) pbits[(size_t)v * n_words + (i >> 3)] = w;
        }
    }
}

// Ancestor filter for V views: the path is read once per node, then checked
// against the P bits of every view in which the node passed.
__global__ void __launch_bounds__(256) banc_kernel(DevTree t, int V, const uint32_t* __restrict__ pbits,
                                                   uint32_t* __restrict__ selbits)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t n_words = t.n_pad >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_words; w += n_warps) {
        const uint32_t n = (w << 5) + lane;
        uint64_t mine = 0;                        // bit v: P in view v
        for (int v = 0; v < V; ++v)
            if ((__ldg(pbits + (size_t)v * n_words + w) >> lane) & 1u) mine |= 1ull << v;
        if (n >= t.n) mine = 0;
        uint64_t keep = mine;
        if (mine) {
            uint32_t a[16];
            for (uint32_t k0 = 0; k0 < t.depth && keep; k0 += 16) {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    a[q] = (k0 + q < t.depth) ? __ldg(t.ap + (size_t)(k0 + q) * t.n_pad + n) : kApPad;
                uint64_t left = keep;
                while (left) {
                    const int v = __ffsll((long long)left) - 1;
                    left &= left - 1;
                    const uint32_t* pv = pbits + (size_t)v * n_words;
                    bool blocked = false;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        if (a[q] == kApPad) break;
                        if ((__ldg(pv + (a[q] >> 5)) >> (a[q] & 31)) & 1u) { blocked = true; break; }
                    }
                    if (blocked) keep &= ~(1ull << v);
                }
                if (a[15] == kApPad) break;
            }
        }
        for (int v = 0; v < V; ++v) {
            const uint32_t b = __ballot_sync(0xffffffffu, (keep >> v) & 1ull);
            if (lane == (uint32_t)(v & 31)) selbits[(size_t)v * n_words + w] = b;
        }
    }
}

// Projection of every selected entry (entry = view * n_pad + node), with the
// pairs counted into global tile ids.
__global__ void __launch_bounds__(kProjThreads) bproject_kernel(
    DevTree t, const DevCamera* __restrict__ cams, int V, const uint32_t* __restrict__ tile_base,
    const uint32_t* __restrict__ sel, float* __restrict__ splat, uint4* __restrict__ foot,
    uint32_t* __restrict__ tile_cnt, FrameState* st)
{
    __shared__ DevCamera s_cam[kMaxBatchViews];
    __shared__ uint32_t s_base[kMaxBatchViews];
    for (int i = threadIdx.x; i < V * (int)(sizeof(DevCamera) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(s_cam)[i] = reinterpret_cast<const uint32_t*>(cams)[i];
    for (int i = threadIdx.x; i < V; i += blockDim.x) s_base[i] = tile_base[i];
    __syncthreads();
    const uint32_t M = st->M;
    const uint32_t n_groups = (M + kProjThreads - 1) / kProjThreads;
    for (uint32_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const uint32_t m = g * kProjThreads + threadIdx.x;
        uint4 f = make_uint4(0, 0, 0, 0);
        uint32_t tiles_x = 1, tbase = 0;
        if (m < M) {
            const uint32_t e = __ldg(sel + m);
            const uint32_t v = e / t.n_pad;
            f = proj::project_one(t, s_cam[v], e - v * t.n_pad, m, splat, foot);
            tiles_x = (uint32_t)s_cam[v].tiles_x;
            tbase = s_base[v];
        }
        warp_count_pairs(f.z, f.x, f.y, tiles_x, tbase, tile_cnt);
    }
}

// Blend every tile of every view; the CTA's view is found by binary search.
__global__ void __launch_bounds__(256) bblend_kernel(const DevCamera* __restrict__ cams, int V,
                                                     const uint32_t* __restrict__ tile_base,
                                                     const unsigned long long* __restrict__ img_off,
                                                     const uint2* __restrict__ ranges,
                                                     const uint32_t* __restrict__ vals,
                                                     const float* __restrict__ splat,
                                                     float* __restrict__ rgb, float* __restrict__ Tout,
                                                     FrameState* st)
{
    __shared__ __align__(128) blendk::HalfSmem H;
    __shared__ DevCamera s_cam;
    const uint32_t gtile = blockIdx.x;
    int lo = 0, hi = V;                            // largest v with tile_base[v] <= gtile
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tile_base + mid) <= gtile) lo = mid;
        else hi = mid;
    }
    const int v = lo;
    for (int i = threadIdx.x; i < (int)(sizeof(DevCamera) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&s_cam)[i] = reinterpret_cast<const uint32_t*>(cams + v)[i];
    __syncthreads();
    const unsigned long long o = __ldg(img_off + v);
    blendk::blend_tile_half(s_cam, gtile - __ldg(tile_base + v), gtile, H, ranges, vals, splat, rgb + 3 * o,
                            Tout ? Tout + o : nullptr, nullptr, st);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_batch_front(const DevTree& t, const DevCamera* cams, int V, uint32_t total_tiles,
                        const uint32_t* tile_base, uint32_t* pbits, uint32_t* selbits, uint32_t* sel,
                        uint32_t sel_cap, float* splat, uint4* foot, uint32_t* tile_cnt, uint32_t* large,
                        unsigned long long* items, unsigned long long* keys, uint32_t* vals,
                        unsigned long long cap, unsigned long long* lb_compact, unsigned long long* lb_scan,
                        uint2* ranges, FrameState* st, int sms, cudaStream_t s)
{
    const uint32_t n_words = t.n_pad >> 5;
    int b0 = (int)((total_tiles + 255) / 256);
    bframe_begin_kernel<<<b0 < 8 ? 8 : b0, 256, 0, s>>>(st, tile_cnt, total_tiles);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bpred_kernel, 256, 0);
    bpred_kernel<<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(t, cams, V, pbits);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, banc_kernel, 256, 0);
    banc_kernel<<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(t, V, pbits, selbits);
    launch_compact(selbits, (uint32_t)((size_t)n_words * V), sel, sel_cap, lb_compact, st,
                   sms * occ_compact(), s);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bproject_kernel, kProjThreads, 0);
    bproject_kernel<<<sms * (occ > 0 ? occ : 1), kProjThreads, 0, s>>>(t, cams, V, tile_base, sel, splat,
                                                                       foot, tile_cnt, st);
    launch_tile_scan(tile_cnt, ranges, total_tiles, large, cap, lb_scan, st, sms * occ_tile_scan(), s);
    launch_scatter_batch(cams, tile_base, t.n_pad, sel, foot, tile_cnt, items, cap, st, sms * occ_scatter(), s);
    launch_segsort(ranges, total_tiles, large, items, keys, vals, st, sms * occ_segsort(), s);
}

void launch_batch_blend(const DevCamera* cams, int V, uint32_t total_tiles, const uint32_t* tile_base,
                        const unsigned long long* img_off, const uint2* ranges, const uint32_t* vals,
                        const float* splat, float* rgb, float* T, FrameState* st, cudaStream_t s)
{
    bblend_kernel<<<total_tiles, 256, 0, s>>>(cams, V, tile_base, img_off, ranges, vals, splat, rgb, T, st);
}

}  // namespace fgs
