// Projection, SH colour, scene-adaptive shrinking and Gaussian-tile key
// emission (§3.1, §3.3) on sm_103a.
//
// One thread per selected Gaussian, 256 per tile, persistent blocks taking
// tiles from a ticket counter.  The radix digit histograms of every emitted key
// (all sort passes) are accumulated here, per block in shared memory.  Each thread computes the splat record (centre,
// conic, log-domain skip threshold, opacity, depth, colour, footprint radius),
// its tile rectangle and pair count; a block scan plus a decoupled look-back
// across tiles gives every Gaussian its first pair slot, so pairs are emitted
// in selection order (the tie-break of the stable (tile | depth) sort).
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

__global__ void __launch_bounds__(kProjThreads) project_emit_kernel(
    DevTree t, DevCamera cam, const uint32_t* __restrict__ sel, float* __restrict__ splat,
    unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals, unsigned long long cap,
    unsigned long long* lookback, FrameState* st)
{
    __shared__ uint32_t s_warp_tot[kProjThreads / 32];
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_hist[kMaxSortPasses][256];   // radix digit histograms of emitted keys
    grid_dep_wait();
    grid_dep_trigger();
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kMaxSortPasses * 256; i += kProjThreads) (&s_hist[0][0])[i] = 0;
    const int passes = cam.sort_passes;
    const uint32_t M = st->M;
    const uint32_t n_tiles = (M + kProjThreads - 1) / kProjThreads;
    const uint32_t tag = st->epoch * 16u + 1u;
    const float fw = (float)cam.tile_w, fh = (float)cam.tile_h;
    const float ftx = (float)cam.tiles_x, fty = (float)cam.tiles_y;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&st->tickets[kTicketProject], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= n_tiles) break;
        const uint32_t m = tile * kProjThreads + tid;
        const bool valid = m < M;
        // ---- 1. everything that decides the pair count (decision-exact binary32)
        uint32_t cnt = 0, n = 0;
        int32_t x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        float mx = 0.0f, my = 0.0f, mz = 0.0f, vz = 0.0f, u = 0.0f, v = 0.0f;
        float A = 0.0f, B = 0.0f, C = 0.0f, radius = 0.0f, a0 = 0.0f, lthr = 0.0f;
        if (valid) {
            n = __ldg(sel + m);
            const size_t np = t.n_pad;
            mx = __ldg(t.mu + n);
            my = __ldg(t.mu + np + n);
            mz = __ldg(t.mu + 2 * np + n);
            float s6[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) s6[q] = __ldg(t.cov + q * np + n);
            a0 = __ldg(t.opacity + n);
            const float ln_a0 = __ldg(t.ln_opacity + n);
            float vx, vy, txtz = 0.0f, tytz = 0.0f;
            camera_space(cam, mx, my, mz, vx, vy, vz);
            const bool inf = frustum_test(cam, vx, vy, vz, txtz, tytz);
            float a = 0.0f, b = 0.0f, c = 0.0f, lam = 0.0f;
            if (inf) ewa_cov2d(cam, vz, txtz, tytz, s6, a, b, c, lam);
            u = fa(fm(cam.fx, fd(vx, vz)), cam.cx);
            v = fa(fm(cam.fy, fd(vy, vz)), cam.cy);
            const float det = fs(fm(a, c), fm(b, b));
            lthr = fs(-5.5412635451584258f, ln_a0);   // -ln 255 - ln alpha0
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
        }
        // ---- 2. block scan of the pair counts, publish the tile aggregate
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
        if (warp == 0) {
            uint32_t prefix = 0;
            if (tile == 0) {
                if (lane == 0) st_lb_u64(lookback + tile, lb_pack(tag, kFlagIncl, total));
            } else {
                if (lane == 0) st_lb_u64(lookback + tile, lb_pack(tag, kFlagAgg, total));
                prefix = warp_lookback(lookback, tile, tag, st, 0x200u);
                if (lane == 0) st_lb_u64(lookback + tile, lb_pack(tag, kFlagIncl, prefix + total));
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (tile == n_tiles - 1) st->n_pairs = (unsigned long long)prefix + total;
            }
        }
        // ---- 3. colour and splat record (overlaps the look-back of warp 0)
        if (valid) {
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
        __syncthreads();
        // ---- 4. warp-cooperative emission: the warp's pairs are numbered 0..wtot-1
        // in (Gaussian, row-major tile) order and written by consecutive lanes.
        // Pair q belongs to the lane whose inclusive count first exceeds q.
        {
            const unsigned long long wfirst = (unsigned long long)s_prefix + off;
            const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - cnt;
            const int32_t rw = x1 - x0;
            const uint32_t dbits = __float_as_uint(vz);
            if (lane == 0 && wtot && wfirst + wtot > cap) set_status(st, kErrCapacity, 0x300u);
            for (uint32_t q0 = 0; q0 < wtot; q0 += 32) {
                const uint32_t q = q0 + lane;
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
                const uint32_t o_d = __shfl_sync(0xffffffffu, dbits, lo);
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
        }
        __syncthreads();
    }
    // flush this block's digit histograms (non-zero bins only)
    for (int i = tid; i < passes * 256; i += kProjThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&st->hist[0][0] + i, c);
    }
}

void launch_project_emit(const DevTree& t, const DevCamera& cam, const uint32_t* sel,
                         float* splat, unsigned long long* keys, uint32_t* vals,
                         unsigned long long cap, unsigned long long* lookback, FrameState* st,
                         int blocks, cudaStream_t s)
{
    if (blocks < 1) blocks = 1;
    launch_pdl(project_emit_kernel, blocks, kProjThreads, 0, s, t, cam, sel, splat, keys, vals, cap,
               lookback, st);
}

int occ_project()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, project_emit_kernel, kProjThreads, 0);
    return b > 0 ? b : 1;
}

}  // namespace fgs
