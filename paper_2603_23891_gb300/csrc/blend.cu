// Per-tile front-to-back alpha blending (Eq. 2) and the KPC / GTC pre-render
// pass of the scene-adaptive shrinking (Eq. 5-7), sm_103a.
//
// One CTA per image tile, one thread per pixel (tile_w * tile_h = 256).  The
// tile's slice of the sorted value list is brought into shared memory in
// chunks of 256 by a TMA bulk copy (cp.async.bulk, completion on an mbarrier;
// the copy starts at the 16-byte boundary at or below the slice and the
// thread index is offset accordingly), then each thread gathers one splat
// record into shared memory and all pixels walk the chunk front to back.
//
// Blend decisions are exact: power, the log-domain skip test, alpha, the
// opacity clamp and the transmittance update use explicitly rounded binary32
// operations and a deterministic exp, so which Gaussians a pixel applies, and
// where it stops, do not depend on the compiler.  Colour accumulation may use
// FMA (it decides nothing).
#include "fgs_internal.cuh"

namespace fgs {

namespace {

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

struct BlendSmem {
    uint32_t vals[kValsSlots];
    float4 g0[kChunk];   // u, v, A, B
    float4 g1[kChunk];   // C, lthr, alpha0, depth
    float4 g2[kChunk];   // r, g, b, radius
    float kpc_w[8][kChunk];   // per-warp partial KPC of each chunk entry
    uint64_t bar;
    int timed_out;
};

// One blend step for a pixel; returns false once the pixel has stopped.
__device__ __forceinline__ void blend_one(const float4& g0, const float4& g1, const float4& g2,
                                          float px, float py, float& T, float3& C, bool& done,
                                          float& w_out)
{
    w_out = 0.0f;
    const float dx = fs(g0.x, px);
    const float dy = fs(g0.y, py);
    const float p1 = fm(fm(g0.z, dx), dx);
    const float p2 = fm(fm(g1.x, dy), dy);
    const float p3 = fm(fm(g0.w, dx), dy);
    const float power = fs(fm(-0.5f, fa(p1, p2)), p3);
    if (power > 0.0f || power < g1.y) return;
    float alpha = fm(g1.z, exp_cw(power));
    alpha = alpha < 0.99f ? alpha : 0.99f;
    const float Tn = fm(T, fs(1.0f, alpha));
    if (Tn < 0.0001f) {
        done = true;
        return;
    }
    const float w = alpha * T;
    C.x = fmaf(g2.x, w, C.x);
    C.y = fmaf(g2.y, w, C.y);
    C.z = fmaf(g2.z, w, C.z);
    w_out = w;
    T = Tn;
}

// Bring chunk [s0, e0) of vals into shared memory.  Returns the offset of s0
// inside the staged copy.  Called by all threads; thread 0 issues the copy.
__device__ __forceinline__ uint32_t stage_vals(BlendSmem& S, const uint32_t* vals, uint32_t s0,
                                               uint32_t e0, uint32_t& phase, FrameState* st)
{
    const uint32_t a0 = s0 & ~3u;
    const uint32_t a1 = (e0 + 3u) & ~3u;
    const uint32_t bytes = (a1 - a0) * 4u;
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&S.bar, bytes);
        tma_bulk_g2s(S.vals, vals + a0, bytes, &S.bar);
        uint64_t spins = 0;
        while (!mbar_try_wait(&S.bar, phase)) {
            if (++spins > kSpinLimit) {
                S.timed_out = 1;
                if (st) set_status(st, kErrTimeout, 0x500u);
                break;
            }
        }
    }
    phase ^= 1u;
    __syncthreads();
    return s0 - a0;
}

}  // namespace

template <bool kKpc>
__global__ void __launch_bounds__(256) blend_kernel(DevCamera cam, const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ vals,
                                                    const float* __restrict__ splat,
                                                    float* __restrict__ rgb, float* __restrict__ Tout,
                                                    float* __restrict__ kpc_out,
                                                    float* __restrict__ G_out, FrameState* st)
{
    __shared__ __align__(128) BlendSmem S;
    __shared__ double s_red[8];
    const uint32_t tile = blockIdx.x;
    const uint32_t tid = threadIdx.x;
    const uint32_t tx = tile % (uint32_t)cam.tiles_x, ty = tile / (uint32_t)cam.tiles_x;
    const int32_t x = (int32_t)(tx * cam.tile_w + (tid & (cam.tile_w - 1)));
    const int32_t y = (int32_t)(ty * cam.tile_h + (tid >> cam.tile_shift_x));
    const bool inside = x < cam.width && y < cam.height;
    const float px = fa((float)x, 0.5f), py = fa((float)y, 0.5f);
    const uint2 rg = ranges[tile];
    const uint32_t M = st->M;
    const uint32_t s = rg.x, e = rg.y;

    if (tid == 0) {
        mbar_init(&S.bar, 1);
        S.timed_out = 0;
    }
    double kpc_acc = 0.0;     // this thread's share of the tile's KPC sum (fixed order)
    __syncthreads();

    float T = 1.0f;
    float3 C = make_float3(0.0f, 0.0f, 0.0f);
    bool done = !inside;
    uint32_t phase = 0;

    for (uint32_t s0 = s; s0 < e; s0 += kChunk) {
        const uint32_t e0 = min(e, s0 + kChunk);
        const uint32_t cnt = e0 - s0;
        const uint32_t off = stage_vals(S, vals, s0, e0, phase, st);
        if (S.timed_out) break;
        if (tid < cnt) {
            uint32_t m = S.vals[off + tid];
            if (m >= M) m = 0;      // only after a failed sort (status already latched)
            const float4* g = reinterpret_cast<const float4*>(splat + (size_t)m * kSplatStride);
            S.g0[tid] = __ldg(g);
            S.g1[tid] = __ldg(g + 1);
            S.g2[tid] = __ldg(g + 2);
        }
        __syncthreads();
        if (!kKpc) {
            for (uint32_t j = 0; j < cnt && !done; ++j) {
                float w;
                blend_one(S.g0[j], S.g1[j], S.g2[j], px, py, T, C, done, w);
            }
        } else {
            const uint32_t lane = tid & 31, warp = tid >> 5;
            for (uint32_t j = 0; j < cnt; ++j) {
                float w = 0.0f;
                if (!done) blend_one(S.g0[j], S.g1[j], S.g2[j], px, py, T, C, done, w);
                // Eq. 5: sum of alpha * T over the tile's pixels for this pair; a
                // butterfly per warp, then the 8 warp partials in order: deterministic
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                if (lane == 0) S.kpc_w[warp][j] = w;
            }
            __syncthreads();
            if (tid < cnt) {
                float k = 0.0f;
#pragma unroll
                for (int w8 = 0; w8 < 8; ++w8) k += S.kpc_w[w8][tid];
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
        rgb[pix] = fmaf(T, cam.bg[0], C.x);
        rgb[hw + pix] = fmaf(T, cam.bg[1], C.y);
        rgb[2 * hw + pix] = fmaf(T, cam.bg[2], C.z);
        if (Tout) Tout[pix] = T;
    }
    if (kKpc) {
        // Eq. 6: G = mean KPC over the tile's pairs; fixed-order block reduction
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kpc_acc += __shfl_xor_sync(0xffffffffu, kpc_acc, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = kpc_acc;
        __syncthreads();
        if (tid == 0) {
            const uint32_t n = e - s;
            double sum = 0.0;
            for (int w8 = 0; w8 < 8; ++w8) sum += s_red[w8];
            G_out[tile] = n > 0 ? (float)(sum / (double)n) : __int_as_float(0x7fc00000);
        }
    }
}

void launch_blend(const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                  const float* splat, float* rgb, float* T, FrameState* st, cudaStream_t s)
{
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    blend_kernel<false><<<n_tiles, 256, 0, s>>>(cam, ranges, vals, splat, rgb, T, nullptr, nullptr,
                                                st);
}

void launch_blend_kpc(const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                      const float* splat, float* kpc, float* G, FrameState* st, cudaStream_t s)
{
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    blend_kernel<true><<<n_tiles, 256, 0, s>>>(cam, ranges, vals, splat, nullptr, nullptr, kpc, G, st);
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
