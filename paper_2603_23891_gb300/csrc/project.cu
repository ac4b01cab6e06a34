// Projection, SH colour, scene-adaptive shrinking and Gaussian-tile key
// emission (§3.1, §3.3) on sm_103a.
//
// Two passes.  project_kernel: one thread per selected Gaussian computes the
// splat record (centre, conic, log-domain skip threshold, opacity, depth,
// colour, footprint radius), its tile rectangle and pair count, and each tile
// of 256 Gaussians its pair total.  emit_kernel: exclusive prefixes of those
// totals give every Gaussian its first pair slot, so pairs are emitted in
// selection order (the tie-break of the stable (tile | depth) sort).
#include "fgs_internal.cuh"

namespace fgs {

namespace {

// Real spherical harmonics (Condon-Shortley phase), Cartesian form, normalisation
// constants from their closed forms: l=0 1/(2 sqrt(pi)); l=1 sqrt(3/(4 pi));
// l=2 sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4; l=3 sqrt(35/(2 pi))/4,
// sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kY00 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.54627421529603959f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.8906114426405538f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011540f;
constexpr float kY3e = 1.4453057213202769f;

// Colour = sum_k Y_k(d) c[k][ch] + 0.5, clamped at 0.  The coefficients are
// streamed as 16-byte loads (node-major, K*3 floats padded to a multiple of 4)
// and accumulated on the fly; element e of the stream is (k, ch) = (e / 3, e % 3).
__device__ __forceinline__ void sh_colour(const float* __restrict__ c, int deg, float x, float y,
                                          float z, float rgb[3])
{
    float Y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = 0.0f;
    Y[0] = kY00;
    if (deg >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (deg >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.0f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (deg >= 3) {
            Y[9] = -kY3a * y * (3.0f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.0f * zz - xx - yy);
            Y[12] = kY3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -kY3c * x * (4.0f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.0f * yy);
        }
    }
    const int K = (deg + 1) * (deg + 1);
    const int nq = (K * 3 + 3) >> 2;
    float acc[3] = {0.5f, 0.5f, 0.5f};
    const float4* c4 = reinterpret_cast<const float4*>(c);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        if (q < nq) {
            const float4 f = __ldg(c4 + q);
            const float e[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int el = 4 * q + r;          // compile-time after unrolling
                if (el < 48) acc[el % 3] = fmaf(Y[el / 3], e[r], acc[el % 3]);
            }
        }
    }
    rgb[0] = fmaxf(acc[0], 0.0f);
    rgb[1] = fmaxf(acc[1], 0.0f);
    rgb[2] = fmaxf(acc[2], 0.0f);
}

__device__ __forceinline__ float clampf(float v, float lo, float hi)
{
    v = v < lo ? lo : v;
    return v > hi ? hi : v;
}

}  // namespace

// Pass 1: one thread per selected Gaussian.  Writes the splat record, a 16-byte
// footprint record {x0, x1, y0, y1 (u16), pair count, depth bits} and, per tile
// of 256 Gaussians, the tile's pair total.  No inter-block dependency.
__global__ void __launch_bounds__(kProjThreads) project_kernel(
    DevTree t, DevCamera cam, const uint32_t* __restrict__ sel, float* __restrict__ splat,
    uint4* __restrict__ foot, uint32_t* __restrict__ tile_total, FrameState* st)
{
    __shared__ uint32_t s_warp_tot[kProjThreads / 32];
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t M = st->M;
    const uint32_t n_tiles = (M + kProjThreads - 1) / kProjThreads;
    const float fw = (float)cam.tile_w, fh = (float)cam.tile_h;
    const float ftx = (float)cam.tiles_x, fty = (float)cam.tiles_y;

    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t m = tile * kProjThreads + tid;
        uint32_t cnt = 0;
        if (m < M) {
            // ---- decision-exact binary32: frustum, EWA covariance, footprint
            const uint32_t n = __ldg(sel + m);
            const size_t np = t.n_pad;
            const float mx = __ldg(t.mu + n), my = __ldg(t.mu + np + n), mz = __ldg(t.mu + 2 * np + n);
            float s6[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) s6[q] = __ldg(t.cov + q * np + n);
            const float a0 = __ldg(t.opacity + n);
            const float ln_a0 = __ldg(t.ln_opacity + n);
            float vx, vy, vz, txtz = 0.0f, tytz = 0.0f;
            camera_space(cam, mx, my, mz, vx, vy, vz);
            const bool inf = frustum_test(cam, vx, vy, vz, txtz, tytz);
            float a = 0.0f, b = 0.0f, c = 0.0f, lam = 0.0f;
            if (inf) ewa_cov2d(cam, vz, txtz, tytz, s6, a, b, c, lam);
            const float u = fa(fm(cam.fx, fd(vx, vz)), cam.cx);
            const float v = fa(fm(cam.fy, fd(vy, vz)), cam.cy);
            const float det = fs(fm(a, c), fm(b, b));
            const float lthr = fs(-5.5412635451584258f, ln_a0);   // -ln 255 - ln alpha0
            float A = 0.0f, B = 0.0f, C = 0.0f, radius = 0.0f;
            int32_t x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            if (inf && det > 0.0f) {
                A = fd(c, det);
                B = fd(-b, det);
                C = fd(a, det);
                // 3-sigma radius, or the radius where alpha0 e^{-r^2/(2 lambda)} = tau,
                // capped at 3 sigma; alpha0 <= tau emits nothing (§3.3)
                float r = fm(3.0f, fsq(lam));
                bool drop = false;
                if (cam.shrink) {
                    const float g = fm(2.0f, fs(ln_a0, cam.ln_tau));
                    if (!(g > 0.0f)) drop = true;
                    else if (g < 9.0f) r = fsq(fm(lam, g));
                }
                if (!drop) {
                    radius = r;
                    const float fx0 = clampf(floorf(fd(fs(u, r), fw)), 0.0f, ftx);
                    const float fx1 = clampf(fa(floorf(fd(fa(u, r), fw)), 1.0f), 0.0f, ftx);
                    const float fy0 = clampf(floorf(fd(fs(v, r), fh)), 0.0f, fty);
                    const float fy1 = clampf(fa(floorf(fd(fa(v, r), fh)), 1.0f), 0.0f, fty);
                    x0 = (int32_t)fx0; x1 = (int32_t)fx1; y0 = (int32_t)fy0; y1 = (int32_t)fy1;
                    if (x1 > x0 && y1 > y0) cnt = (uint32_t)((x1 - x0) * (y1 - y0));
                }
            }
            foot[m] = make_uint4((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16),
                                 cnt, __float_as_uint(vz));
            // ---- colour (FMA allowed: decides nothing)
            float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
            const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= il; dy *= il; dz *= il;
            float rgb[3];
            sh_colour(t.sh + (size_t)n * t.sh_stride, (int)t.sh_degree, dx, dy, dz, rgb);
            float4* out = reinterpret_cast<float4*>(splat + (size_t)m * kSplatStride);
            out[0] = make_float4(u, v, A, B);
            out[1] = make_float4(C, lthr, a0, vz);
            out[2] = make_float4(rgb[0], rgb[1], rgb[2], radius);
        }
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
}

// Pass 2: pair slots and key emission.  Block b takes kEmitTiles consecutive
// Gaussian tiles; its first slot is the sum of all earlier tile totals (a block
// reduction, no waiting on other blocks).  Within a tile a block scan orders
// the Gaussians, and each warp writes its pairs with consecutive lanes on
// consecutive slots.  The radix digit histograms of all sort passes are
// accumulated here, per block in shared memory.
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
                        for (int p = 0; p < passes; ++p)
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
    for (int i = tid; i < passes * 256; i += kProjThreads) {
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
