// Per-tile front-to-back alpha blending (Eq. 2) and the KPC / GTC pre-render
// pass of the scene-adaptive shrinking (Eq. 5-7), sm_103a.
//
// One CTA per image tile, one thread per pixel (tile_w * tile_h = 256); each
// warp covers an 8 x 4 (or 4 x 8) pixel block.  The tile's slice of the sorted
// value list is brought into shared memory in chunks of 256 by a TMA bulk copy
// (cp.async.bulk, completion on an mbarrier; the copy starts at the 16-byte
// boundary at or below the slice and the index is offset accordingly); in the
// forward two buffers alternate, the next chunk's copy landing while the
// current chunk is walked.  Each thread then gathers one splat record into
// shared memory and computes which pixel blocks the Gaussian can reach.  The forward culls per 4 x 4 half-block
// (each warp's two halves walk their own ordered lists in lockstep, testing in
// groups of 32 entries and then applying each lane's hits); the KPC pass culls
// per warp and walks one entry at a time, reducing alpha * T across the warp.
//
// Blend decisions are exact: power, the log-domain skip test, alpha, the
// opacity clamp and the transmittance update use explicitly rounded binary32
// operations and a deterministic exp, so which Gaussians a pixel applies, and
// where it stops, do not depend on the compiler.  The culling only drops
// Gaussians that every pixel of the block would skip.  Colour accumulation may
// use FMA (it decides nothing).
#include "blend_impl.cuh"

namespace fgs {

using blendk::BlendSmem;

template <bool kKpc, bool kCount = false, bool kKeep = false>
__global__ void __launch_bounds__(256) blend_kernel(DevCamera cam, const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ vals,
                                                    const float* __restrict__ splat,
                                                    float* __restrict__ rgb, float* __restrict__ Tout,
                                                    uint2* __restrict__ keep,
                                                    float* __restrict__ kpc_out,
                                                    float* __restrict__ G_out, FrameState* st)
{
    if constexpr (kKpc) {
        __shared__ __align__(128) BlendSmem<true> S;
        __shared__ double s_red[8];
        grid_dep_wait();
        grid_dep_trigger();
        blendk::blend_tile_kpc(cam, blockIdx.x, S, s_red, ranges, vals, splat, kpc_out, G_out, st);
    } else {
        __shared__ __align__(128) blendk::HalfSmem H;
        grid_dep_wait();
        grid_dep_trigger();
        blendk::blend_tile_half<kCount, kKeep>(cam, blockIdx.x, blockIdx.x, H, ranges, vals, splat, rgb,
                                               Tout, keep, st);
    }
}

void launch_blend(const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                  const float* splat, float* rgb, float* T, uint2* keep, FrameState* st, bool count,
                  cudaStream_t s)
{
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    float* const nf = nullptr;
    if (count)
        launch_pdl(blend_kernel<false, true>, n_tiles, 256, 0, s, cam, ranges, vals, splat, rgb, T, keep,
                   nf, nf, st);
    else if (keep)
        launch_pdl(blend_kernel<false, false, true>, n_tiles, 256, 0, s, cam, ranges, vals, splat, rgb, T,
                   keep, nf, nf, st);
    else
        launch_pdl(blend_kernel<false>, n_tiles, 256, 0, s, cam, ranges, vals, splat, rgb, T, keep, nf, nf,
                   st);
}

void launch_blend_kpc(const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                      const float* splat, float* kpc, float* G, FrameState* st, cudaStream_t s)
{
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    launch_pdl(blend_kernel<true>, n_tiles, 256, 0, s, cam, ranges, vals, splat, (float*)nullptr,
               (float*)nullptr, (uint2*)nullptr, kpc, G, st);
}

__global__ void eval_exp_kernel(const float* __restrict__ x, float* __restrict__ y, uint64_t n)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = exp_cw(x[i]);
}

void launch_eval_exp(const float* x, float* y, uint64_t n, cudaStream_t s)
{
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    eval_exp_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
}

}  // namespace fgs
