// Differentiable form of the render path: parameter preparation, and the
// hand-written backward of blending (Eq. 2), EWA projection and SH colour.
//
// Selection, tile rectangles and every skip / stop decision of blending are
// held fixed (a discrete cut), as in 3DGS training.  Per-Gaussian parameters:
// mean mu, log-scale s, quaternion q (any norm), opacity logit l, SH
// coefficients; Sigma = R(q/|q|) diag(e^{2s}) R^T, alpha0 = sigmoid(l).
//
// blend_bwd_kernel recomputes each pixel's final transmittance and stop
// position by a front-to-back walk over its tile with the forward's exact
// decisions (or, after a FGS_RENDER_KEEP forward, reads the 8 bytes per pixel
// the forward kept), then walks the tile back to front, recovering T before
// each Gaussian as T / (1 - alpha) and accumulating the colour behind it;
// chunks past the last stop of the tile are never loaded.  Gradients with respect to the splat record (u, v,
// conic A B C, alpha0, colour) are reduced per warp (a transposed reduction:
// 12 shuffles for 9 values) and added per Gaussian; project_bwd_kernel then
// applies the chain rule to the parameters.
#include "blend_impl.cuh"

#include <type_traits>
#include "project_impl.cuh"

namespace fgs {

constexpr int kGS = 12;   // floats per splat gradient: u v A B C a0 r g b (3 spare)

// ---------------------------------------------------------------------------
// parameters -> binary32 attributes, in one fixed operation order (no fused
// operations), so that the selection and blending decisions taken on them are
// reproducible bit for bit by any IEEE binary32 implementation of that order
// ---------------------------------------------------------------------------

// ln x for positive normal x: x = 2^e m, m in [sqrt(1/2), sqrt(2)] from the
// exponent bits; ln m = 2 atanh(s), s = (m - 1) / (m + 1), by the odd series
// 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9) (|s| < 0.172, truncation below 1e-9
// relative; Abramowitz & Stegun 4.1.27); plus e ln 2.
__device__ __forceinline__ float ln_cw(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421356f) {
        m = fm(m, 0.5f);
        e += 1;
    }
    const float s = fd(fs(m, 1.0f), fa(m, 1.0f));
    const float s2 = fm(s, s);
    float p = 0.111111111f;
    p = fa(fm(p, s2), 0.142857143f);
    p = fa(fm(p, s2), 0.2f);
    p = fa(fm(p, s2), 0.333333333f);
    p = fa(fm(p, s2), 1.0f);
    return fa(fm((float)e, 0.693147182f), fm(fm(2.0f, s), p));
}

struct ParamPtrs {
    const float* mu;          // [3][n]
    const float* log_scale;   // [3][n]
    const float* quat;        // [4][n] (w, x, y, z), any non-zero norm
    const float* logit;       // [n]
    const float* sh;          // [n][K][3]
    uint32_t n;
};

constexpr float kLogitMax = 80.0f;

// Sigma = R(q/|q|) diag(e^{2 s}) R(q/|q|)^T (6 upper-triangle entries, order
// xx xy xz yy yz zz) and the pieces the backward needs.
__device__ __forceinline__ void sigma_from(const ParamPtrs& p, uint32_t n, float cov[6], float R[9],
                                           float s2[3], float qh[4], float& qn)
{
    const size_t N = p.n;
    const float w = p.quat[n], x = p.quat[N + n], y = p.quat[2 * N + n], z = p.quat[3 * N + n];
    qn = fsq(fa(fa(fa(fm(w, w), fm(x, x)), fm(y, y)), fm(z, z)));
    const float qw = fd(w, qn), qx = fd(x, qn), qy = fd(y, qn), qz = fd(z, qn);
    qh[0] = qw; qh[1] = qx; qh[2] = qy; qh[3] = qz;
    R[0] = fs(1.0f, fm(2.0f, fa(fm(qy, qy), fm(qz, qz))));
    R[1] = fm(2.0f, fs(fm(qx, qy), fm(qw, qz)));
    R[2] = fm(2.0f, fa(fm(qx, qz), fm(qw, qy)));
    R[3] = fm(2.0f, fa(fm(qx, qy), fm(qw, qz)));
    R[4] = fs(1.0f, fm(2.0f, fa(fm(qx, qx), fm(qz, qz))));
    R[5] = fm(2.0f, fs(fm(qy, qz), fm(qw, qx)));
    R[6] = fm(2.0f, fs(fm(qx, qz), fm(qw, qy)));
    R[7] = fm(2.0f, fa(fm(qy, qz), fm(qw, qx)));
    R[8] = fs(1.0f, fm(2.0f, fa(fm(qx, qx), fm(qy, qy))));
#pragma unroll
    for (int k = 0; k < 3; ++k) s2[k] = exp_cw(fm(2.0f, p.log_scale[k * N + n]));
    constexpr int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int i = ij[e][0], j = ij[e][1];
        cov[e] = fa(fa(fm(fm(R[3 * i], s2[0]), R[3 * j]), fm(fm(R[3 * i + 1], s2[1]), R[3 * j + 1])),
                    fm(fm(R[3 * i + 2], s2[2]), R[3 * j + 2]));
    }
}

__device__ __forceinline__ float clamp_logit(float l)
{
    return l < -kLogitMax ? -kLogitMax : (l > kLogitMax ? kLogitMax : l);
}

// Parameters -> the tree attributes the frame kernels read: mu, Sigma,
// alpha0 = sigmoid(l), ln alpha0 = -ln(1 + e^{-l}) (l clamped to [-80, 80]), SH.
__global__ void __launch_bounds__(256) prep_params_kernel(DevTree t, ParamPtrs p)
{
    float* mu = const_cast<float*>(t.mu);
    float* cov = const_cast<float*>(t.cov);
    float* op = const_cast<float*>(t.opacity);
    float* lop = const_cast<float*>(t.ln_opacity);
    const size_t np = t.n_pad, N = p.n;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < p.n; n += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) mu[k * np + n] = p.mu[k * N + n];
        float c6[6], R[9], s2[3], qh[4], qn;
        sigma_from(p, n, c6, R, s2, qh, qn);
#pragma unroll
        for (int k = 0; k < 6; ++k) cov[k * np + n] = c6[k];
        const float den = fa(1.0f, exp_cw(-clamp_logit(p.logit[n])));
        const float a0 = fd(1.0f, den), la0 = -ln_cw(den);
        op[n] = a0;
        lop[n] = la0;
        float4* attr = const_cast<float4*>(t.attr) + 3 * (size_t)n;
        attr[0] = make_float4(p.mu[n], p.mu[N + n], p.mu[2 * N + n], a0);
        attr[1] = make_float4(c6[0], c6[1], c6[2], c6[3]);
        attr[2] = make_float4(c6[4], c6[5], la0, 0.0f);
    }
}

// SH coefficients [n][K3] -> the tree's rows of sh_stride floats, one flat
// coalesced pass over the source (K3 a compile-time constant: the division is
// a multiply).
template <int kDeg>
__global__ void __launch_bounds__(256) prep_sh_kernel(DevTree t, const float* __restrict__ src)
{
    constexpr uint64_t K3 = (kDeg + 1) * (kDeg + 1) * 3;
    float* sh = const_cast<float*>(t.sh);
    const uint64_t total = (uint64_t)t.n * K3;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t n = i / K3;
        sh[n * t.sh_stride + (i - n * K3)] = __ldg(src + i);
    }
}

// ---------------------------------------------------------------------------
// blend backward
// ---------------------------------------------------------------------------
// Shared memory of the blend backward: the forward's half-block walk (used to
// recompute each pixel's final T and stop position) and the back-to-front
// gradient walk over half-block lists, one after the other.
struct BwdWalkSmem {
    uint32_t vals[blendk::kValsSlots];
    float4 g0[blendk::kChunk];                  // u, v, A', B'
    float4 g1[blendk::kChunk];                  // C', lthr, alpha0, depth
    float4 g2[blendk::kChunk];                  // r, g, b, radius
    uint32_t m[blendk::kChunk];                 // selected rank of each chunk entry
    uint16_t hmask[blendk::kChunk];
    alignas(16) uint8_t hl[blendk::kHalfBlocks][blendk::kChunk];
    uint32_t hlim[blendk::kHalfBlocks];         // last stop position of each half-block
    uint64_t bar;
    int timed_out;
};
union BwdSmem {
    blendk::HalfSmem fwd;
    BwdWalkSmem bwd;
};
__device__ __forceinline__ BwdWalkSmem& walk_smem(BwdSmem& b) { return b.bwd; }
__device__ __forceinline__ BwdWalkSmem& walk_smem(BwdWalkSmem& b) { return b; }

// Sum over each half-warp (16 lanes) of v[0..8], scattered: on return the lane
// given by half_component() holds its half's sum of that component.  Recursive
// halving within the half (xor 8, 4, 2, 1 split the value set): 11 shuffles.
__device__ __forceinline__ float half_reduce9(const float v[9], uint32_t lane)
{
    const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2, b0 = lane & 1;
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = v[i], hi = (5 + i < 9) ? v[5 + i] : 0.0f;
        a[i] = (b3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8);
    }
    float b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float lo = a[i], hi = (3 + i < 5) ? a[3 + i] : 0.0f;
        b[i] = (b2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b2 ? lo : hi, 4);
    }
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float lo = b[i], hi = (2 + i < 3) ? b[2 + i] : 0.0f;
        c[i] = (b1 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b1 ? lo : hi, 2);
    }
    return (b0 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b0 ? c[0] : c[1], 1);
}

// Component whose half sum half_reduce9 leaves in this lane (-1: padding).
__device__ __forceinline__ int half_component(uint32_t lane)
{
    const int pb = 2 * ((lane >> 1) & 1) + (lane & 1);
    const int pa = 3 * ((lane >> 2) & 1) + pb;
    const int comp = 5 * ((lane >> 3) & 1) + pa;
    return (pb < 3 && pa < 5 && comp < 9) ? comp : -1;
}

// kKept: the forward kept {final T, stop} per pixel (FGS_RENDER_KEEP) in keep.
// Otherwise the forward's own half-block walk runs first, without colour, and
// writes them there.  Then the tile is walked back to front over half-block
// lists (a 4x4 half-warp tests only the Gaussians whose threshold box meets
// it, as in the forward), the two halves of a warp in lockstep, each from its
// list's last entry before its last stop.
template <bool kKept>
__global__ void __launch_bounds__(256) blend_bwd_kernel(DevCamera cam, const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals,
                                                        const float* __restrict__ splat,
                                                        uint2* __restrict__ keep,
                                                        const float* __restrict__ dL_drgb,
                                                        float* __restrict__ gsplat, FrameState* st)
{
    // (with kept state the forward walk's shared memory is not needed)
    __shared__ __align__(128) typename std::conditional<kKept, BwdWalkSmem, BwdSmem>::type B;
    const uint32_t tile = blockIdx.x;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if constexpr (!kKept) {
        blendk::blend_tile_half<false, true>(cam, tile, tile, B.fwd, ranges, vals, splat, nullptr, nullptr,
                                            keep, st);
        __syncthreads();
        if (B.fwd.timed_out) return;
    }
    BwdWalkSmem& S = walk_smem(B);
    const int32_t tx0 = (int32_t)(tile % (uint32_t)cam.tiles_x) * cam.tile_w;
    const int32_t ty0 = (int32_t)(tile / (uint32_t)cam.tiles_x) * cam.tile_h;
    int32_t wx0, wy0;
    blendk::warp_origin(cam, tx0, ty0, warp, wx0, wy0);
    const uint32_t half = lane >> 4, q = lane & 15u;
    const bool wide = cam.warp_shift == 3;
    const int32_t x = wx0 + (int32_t)(q & 3u) + (wide ? 4 * (int32_t)half : 0);
    const int32_t y = wy0 + (int32_t)(q >> 2) + (wide ? 0 : 4 * (int32_t)half);
    const uint32_t hb = ((uint32_t)(y - ty0) >> 2 << (cam.tile_shift_x - 2)) | ((uint32_t)(x - tx0) >> 2);
    const uint32_t hb0 = __shfl_sync(0xffffffffu, hb, 0), hb1 = __shfl_sync(0xffffffffu, hb, 16);
    const bool inside = x < cam.width && y < cam.height;
    const float px = fa((float)x, 0.5f), py = fa((float)y, 0.5f);
    const uint2 rg = ranges[tile];
    const uint32_t M = st->M;
    const uint32_t s = rg.x;
    const int comp = half_component(lane);
    const uint32_t lt = (1u << lane) - 1u;

    // this pixel's forward outcome: final T, stop position, and dL/dC
    float T = 1.0f;
    uint32_t lim = s;
    float dC[3] = {0.0f, 0.0f, 0.0f};
    if (inside) {
        const size_t hw = (size_t)cam.width * cam.height, pix = (size_t)y * cam.width + x;
        const uint2 kp = keep[pix];
        T = __uint_as_float(kp.x);
        lim = kp.y;
        dC[0] = __ldg(dL_drgb + pix);
        dC[1] = __ldg(dL_drgb + hw + pix);
        dC[2] = __ldg(dL_drgb + 2 * hw + pix);
    }
    // each half-block's last stop position; the tile's bounds the chunks
    const uint32_t hmax = max(lim, __shfl_xor_sync(0xffffffffu, lim, 8));
    const uint32_t hmax2 = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, 4));
    const uint32_t hmax3 = max(hmax2, __shfl_xor_sync(0xffffffffu, hmax2, 2));
    const uint32_t hlim = max(hmax3, __shfl_xor_sync(0xffffffffu, hmax3, 1));
    if (q == 0) S.hlim[hb] = hlim;
    if (tid == 0) {
        blendk::mbar_init(&S.bar, 1);
        S.timed_out = 0;
    }
    __syncthreads();
    uint32_t e = S.hlim[0];
#pragma unroll
    for (int h = 1; h < blendk::kHalfBlocks; ++h) e = max(e, S.hlim[h]);
    e = min(e, rg.y);                    // no pixel of the tile reaches past e
    const uint32_t hlim0 = S.hlim[hb0], hlim1 = S.hlim[hb1];

    float Bk[3] = {cam.bg[0] * T, cam.bg[1] * T, cam.bg[2] * T};   // colour behind, absolute
    float Tc = T;                                                    // transmittance after
    if (e <= s) return;
    uint32_t phase = 0;
    const uint32_t n_chunks = (e - s + blendk::kChunk - 1) / blendk::kChunk;
    for (int c = (int)n_chunks - 1; c >= 0; --c) {
        const uint32_t s0 = s + (uint32_t)c * blendk::kChunk, e0 = min(e, s0 + blendk::kChunk);
        const uint32_t cnt = e0 - s0;
        const uint32_t off = blendk::stage_vals(S.vals, &S.bar, &S.timed_out, vals, s0, e0, phase, st);
        if (S.timed_out) return;
        if (tid < cnt) {
            uint32_t m = S.vals[off + tid];
            if (m >= M) m = 0;
            const float4* g = reinterpret_cast<const float4*>(splat + (size_t)m * kSplatStride);
            const float4 a = __ldg(g), b = __ldg(g + 1);
            blendk::put_coeffs(S.g0[tid], S.g1[tid], a, b);
            S.g2[tid] = __ldg(g + 2);
            S.hmask[tid] = (uint16_t)blendk::half_mask(cam, tx0, ty0, a.x, a.y, a.z, a.w, b.x, b.y);
            S.m[tid] = m;
        }
        __syncthreads();
        // this warp's two half-block lists of the chunk entries before their last stops
        uint32_t n0 = 0, n1 = 0;
        for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t hm = j < cnt ? (uint32_t)S.hmask[j] : 0u;
            const bool in0 = ((hm >> hb0) & 1u) && s0 + j < hlim0;
            const bool in1 = ((hm >> hb1) & 1u) && s0 + j < hlim1;
            const uint32_t b0 = __ballot_sync(0xffffffffu, in0);
            const uint32_t b1 = __ballot_sync(0xffffffffu, in1);
            if (in0) S.hl[hb0][n0 + __popc(b0 & lt)] = (uint8_t)j;
            if (in1) S.hl[hb1][n1 + __popc(b1 & lt)] = (uint8_t)j;
            n0 += __popc(b0);
            n1 += __popc(b1);
        }
        __syncwarp();
        const uint32_t nmax = max(n0, n1);
        const uint32_t nh = half ? n1 : n0;
        const uint8_t* myl = S.hl[hb];
        // step k: each half takes its entry k - (nmax - nh), the lists' ends aligned
        for (int k = (int)nmax - 1; k >= 0; --k) {
            const int i = k - (int)(nmax - nh);
            const bool valid = i >= 0;
            const uint32_t j = valid ? myl[i] : 0u;
            // branch-free: every lane evaluates; the lanes whose pixel applied the
            // Gaussian in the forward (same decisions) contribute, the others add 0
            const float4 g0 = S.g0[j];
            const float4 g1 = S.g1[j];
            const float dx = fs(g0.x, px), dy = fs(g0.y, py);
            const float power = blendk::power_of(g0.z, g0.w, g1.x, dx, dy);
            const bool hit = valid && s0 + j < lim && !(power > 0.0f || power < g1.y);
            const uint32_t hb_any = __ballot_sync(0xffffffffu, hit);
            if (!hb_any) continue;
            const float ex = exp_nonpos(fminf(power, 0.0f));
            const float raw = fm(g1.z, ex);
            const bool clamped = !(raw < 0.99f);
            const float alpha = hit ? (clamped ? 0.99f : raw) : 0.0f;
            const float4 g2 = S.g2[j];
            const float iom = __frcp_rn(1.0f - alpha);              // decides nothing
            const float Tb = Tc * iom;                               // transmittance before
            const float w = alpha * Tb;
            const float galpha = hit ? dC[0] * (g2.x * Tb - Bk[0] * iom) + dC[1] * (g2.y * Tb - Bk[1] * iom) +
                                       dC[2] * (g2.z * Tb - Bk[2] * iom)
                                     : 0.0f;
            Bk[0] += g2.x * w;
            Bk[1] += g2.y * w;
            Bk[2] += g2.z * w;
            Tc = Tb;
            float g[9];
            g[6] = w * dC[0];
            g[7] = w * dC[1];
            g[8] = w * dC[2];
            const float gpow = clamped ? 0.0f : galpha * alpha;     // d alpha / d power = alpha
            g[5] = clamped ? 0.0f : galpha * ex;                   // d alpha / d alpha0 = e^power
            g[2] = -0.5f * dx * dx * gpow;                         // A
            g[3] = -dx * dy * gpow;                                // B
            g[4] = -0.5f * dy * dy * gpow;                         // C
            // d power / du = -(A dx + B dy) = 2 A' dx + B' dy, likewise for v
            g[0] = gpow * (2.0f * g0.z * dx + g0.w * dy);          // u
            g[1] = gpow * (2.0f * g1.x * dy + g0.w * dx);          // v
            const float v = half_reduce9(g, lane);
            const bool my_half_hit = ((hb_any >> (half << 4)) & 0xFFFFu) != 0u;
            if (comp >= 0 && my_half_hit) atomicAdd(gsplat + (size_t)S.m[j] * kGS + comp, v);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// projection / SH backward (one thread per selected Gaussian)
// ---------------------------------------------------------------------------
namespace {

// Real SH basis (Cartesian form, degree kDeg <= 3) and its partial derivatives
// in (x, y, z), treating the three as independent.
template <int kDeg>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float Y[16], float dY[16][3])
{
    using namespace proj;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.0f;
        dY[k][0] = dY[k][1] = dY[k][2] = 0.0f;
    }
    Y[0] = kY00;
    if (kDeg < 1) return;
    Y[1] = -kY1 * y; dY[1][1] = -kY1;
    Y[2] = kY1 * z;  dY[2][2] = kY1;
    Y[3] = -kY1 * x; dY[3][0] = -kY1;
    if (kDeg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;                 dY[4][0] = kY2a * y;           dY[4][1] = kY2a * x;
    Y[5] = -kY2a * y * z;                dY[5][1] = -kY2a * z;          dY[5][2] = -kY2a * y;
    Y[6] = kY2b * (2.0f * zz - xx - yy); dY[6][0] = -2.0f * kY2b * x;   dY[6][1] = -2.0f * kY2b * y;
    dY[6][2] = 4.0f * kY2b * z;
    Y[7] = -kY2a * x * z;                dY[7][0] = -kY2a * z;          dY[7][2] = -kY2a * x;
    Y[8] = kY2c * (xx - yy);             dY[8][0] = 2.0f * kY2c * x;    dY[8][1] = -2.0f * kY2c * y;
    if (kDeg < 3) return;
    Y[9] = -kY3a * y * (3.0f * xx - yy);
    dY[9][0] = -6.0f * kY3a * x * y;
    dY[9][1] = -kY3a * (3.0f * xx - 3.0f * yy);
    Y[10] = kY3b * x * y * z;
    dY[10][0] = kY3b * y * z;
    dY[10][1] = kY3b * x * z;
    dY[10][2] = kY3b * x * y;
    Y[11] = -kY3c * y * (4.0f * zz - xx - yy);
    dY[11][0] = 2.0f * kY3c * x * y;
    dY[11][1] = -kY3c * (4.0f * zz - xx - 3.0f * yy);
    dY[11][2] = -8.0f * kY3c * y * z;
    Y[12] = kY3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    dY[12][0] = -6.0f * kY3d * x * z;
    dY[12][1] = -6.0f * kY3d * y * z;
    dY[12][2] = kY3d * (6.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -kY3c * x * (4.0f * zz - xx - yy);
    dY[13][0] = -kY3c * (4.0f * zz - 3.0f * xx - yy);
    dY[13][1] = 2.0f * kY3c * x * y;
    dY[13][2] = -8.0f * kY3c * x * z;
    Y[14] = kY3e * z * (xx - yy);
    dY[14][0] = 2.0f * kY3e * x * z;
    dY[14][1] = -2.0f * kY3e * y * z;
    dY[14][2] = kY3e * (xx - yy);
    Y[15] = -kY3a * x * (xx - 3.0f * yy);
    dY[15][0] = -kY3a * (3.0f * xx - 3.0f * yy);
    dY[15][1] = 6.0f * kY3a * x * y;
}

}  // namespace

struct GradPtrs {
    float* mu;          // [3][n]
    float* log_scale;   // [3][n]
    float* quat;        // [4][n]
    float* logit;       // [n]
    float* sh;          // [n][K][3]
};

// Chain rule for selected Gaussian m (node sel[m]): splat gradient -> mean,
// log-scale, quaternion, logit, SH.  Each node appears once in the selection,
// so plain stores (or read-modify-writes when accumulating) need no atomics.
//
// Each warp takes 32 consecutive selected Gaussians per iteration, one per
// lane.  Their SH rows (3 K floats each, contiguous per node) are staged in
// shared memory with coalesced asynchronous copies, and the SH gradient rows
// leave the same way; the row stride 3 K + 1 is odd, so lane l reading row l, element k hits
// bank (l (3 K + 1) + k) mod 32, a different bank for every lane.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(blendk::smem_addr(smem)), "l"(gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int kPbWarps = 2;   // warps per projection-backward block

template <int kDeg, bool kAccumulate>
__global__ void __launch_bounds__(kPbWarps * 32, 16 / kPbWarps) project_bwd_kernel(DevTree t, DevCamera cam, ParamPtrs p,
                                                          const uint32_t* __restrict__ sel,
                                                          const float* __restrict__ gsplat,
                                                          GradPtrs gr, const FrameState* st)
{
    constexpr int K = (kDeg + 1) * (kDeg + 1);
    constexpr int K3 = 3 * K, RS = K3 + 1;
    __shared__ float s_rows[kPbWarps][32 * RS];
    __shared__ float s_olds[kAccumulate ? kPbWarps : 1][kAccumulate ? 32 * RS : 1];
    const uint32_t M = st->M;
    const size_t N = p.n;
    const float* W = cam.R;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* rows = s_rows[warp];
    float* olds = s_olds[kAccumulate ? warp : 0];
    float* row = rows + lane * RS;
    for (uint32_t base = (blockIdx.x * kPbWarps + warp) * 32; base < M; base += gridDim.x * kPbWarps * 32) {
        const uint32_t m = base + lane;
        const bool act = m < M;
        const uint32_t n = act ? sel[m] : sel[base];
        // stage the warp's SH rows (and, accumulating, their current gradient
        // rows) with asynchronous copies: element i * 32 + lane of the 32 x K3
        // block, all in flight at once, no registers held
#pragma unroll
        for (int i = 0; i < K3; ++i) {
            const uint32_t idx = (uint32_t)i * 32u + lane, r = idx / K3, k = idx - r * K3;
            const uint32_t nr = __shfl_sync(0xffffffffu, n, r);
            cp_async4(rows + r * RS + k, p.sh + (size_t)nr * K3 + k);
            if (kAccumulate && base + r < M) cp_async4(olds + r * RS + k, gr.sh + (size_t)nr * K3 + k);
        }
        cp_async_wait_all();
        __syncwarp();
        const float* gs = gsplat + (size_t)(act ? m : base) * kGS;
        const float gu = gs[0], gv = gs[1], gA = gs[2], gB = gs[3], gC = gs[4], ga0 = gs[5];
        const float gcol[3] = {gs[6], gs[7], gs[8]};
        const float mu[3] = {p.mu[n], p.mu[N + n], p.mu[2 * N + n]};
        // camera space (the Gaussian passed the frustum test, so the tangent
        // clamp of the EWA Jacobian is inactive)
        const float x = W[0] * mu[0] + W[1] * mu[1] + W[2] * mu[2] + cam.t[0];
        const float y = W[3] * mu[0] + W[4] * mu[1] + W[5] * mu[2] + cam.t[1];
        const float z = W[6] * mu[0] + W[7] * mu[1] + W[8] * mu[2] + cam.t[2];
        const float iz = 1.0f / z, iz2 = iz * iz;
        float c6[6], Rq[9], s2[3], qh[4], qn;
        sigma_from(p, n, c6, Rq, s2, qh, qn);
        const float Sg[3][3] = {{c6[0], c6[1], c6[2]}, {c6[1], c6[3], c6[4]}, {c6[2], c6[4], c6[5]}};
        const float J[2][3] = {{cam.fx * iz, 0.0f, -cam.fx * x * iz2}, {0.0f, cam.fy * iz, -cam.fy * y * iz2}};
        float Mm[2][3], MS[2][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Mm[i][j] = J[i][0] * W[j] + J[i][1] * W[3 + j] + J[i][2] * W[6 + j];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) MS[i][j] = Mm[i][0] * Sg[0][j] + Mm[i][1] * Sg[1][j] + Mm[i][2] * Sg[2][j];
        const float a = MS[0][0] * Mm[0][0] + MS[0][1] * Mm[0][1] + MS[0][2] * Mm[0][2] + 0.3f;
        const float b = MS[0][0] * Mm[1][0] + MS[0][1] * Mm[1][1] + MS[0][2] * Mm[1][2];
        const float c = MS[1][0] * Mm[1][0] + MS[1][1] * Mm[1][1] + MS[1][2] * Mm[1][2] + 0.3f;
        const float det = a * c - b * b, id2 = 1.0f / (det * det);
        // conic (A, B, C) = (c, -b, a) / det  ->  Sigma_2D entries (a, b, c)
        const float ga = (gA * (-c * c) + gB * (b * c) + gC * (-b * b)) * id2;
        const float gb = (gA * (2.0f * b * c) - gB * (det + 2.0f * b * b) + gC * (2.0f * a * b)) * id2;
        const float gc = (gA * (-b * b) + gB * (a * b) + gC * (-a * a)) * id2;
        const float G2[2][2] = {{ga, 0.5f * gb}, {0.5f * gb, gc}};
        // Sigma_2D = M Sigma M^T: dL/dSigma = M^T G2 M, dL/dM = 2 G2 M Sigma
        float GS[3][3], GM[2][3], GJ[2][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float v = 0.0f;
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int l = 0; l < 2; ++l) v += Mm[k][i] * G2[k][l] * Mm[l][j];
                GS[i][j] = v;
            }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) GM[i][j] = 2.0f * (G2[i][0] * MS[0][j] + G2[i][1] * MS[1][j]);
        // M = J W
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                GJ[i][k] = GM[i][0] * W[3 * k] + GM[i][1] * W[3 * k + 1] + GM[i][2] * W[3 * k + 2];
        // (u, v) and J as functions of the camera-space centre
        const float gx = gu * cam.fx * iz - GJ[0][2] * cam.fx * iz2;
        const float gy = gv * cam.fy * iz - GJ[1][2] * cam.fy * iz2;
        const float gz = -(gu * cam.fx * x + gv * cam.fy * y) * iz2 - (GJ[0][0] * cam.fx + GJ[1][1] * cam.fy) * iz2 +
                         2.0f * (GJ[0][2] * cam.fx * x + GJ[1][2] * cam.fy * y) * iz2 * iz;
        float gmu[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) gmu[j] = W[j] * gx + W[3 + j] * gy + W[6 + j] * gz;
        // Sigma = R diag(s2) R^T: dL/dR = 2 GS R diag(s2), dL/ds_k = 2 s2_k (R^T GS R)_kk
        float G[9], gls[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                G[3 * i + k] = 2.0f * (GS[i][0] * Rq[k] + GS[i][1] * Rq[3 + k] + GS[i][2] * Rq[6 + k]) * s2[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float v = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) v += Rq[3 * i + k] * GS[i][j] * Rq[3 * j + k];
            gls[k] = 2.0f * s2[k] * v;
        }
        // R(q/|q|): derivatives of the nine entries in the unit quaternion
        const float w_ = qh[0], x_ = qh[1], y_ = qh[2], z_ = qh[3];
        float gq[4];
        gq[0] = 2.0f * (-z_ * G[1] + y_ * G[2] + z_ * G[3] - x_ * G[5] - y_ * G[6] + x_ * G[7]);
        gq[1] = 2.0f * (y_ * G[1] + z_ * G[2] + y_ * G[3] - 2.0f * x_ * G[4] - w_ * G[5] + z_ * G[6] +
                        w_ * G[7] - 2.0f * x_ * G[8]);
        gq[2] = 2.0f * (-2.0f * y_ * G[0] + x_ * G[1] + w_ * G[2] + x_ * G[3] + z_ * G[5] - w_ * G[6] +
                        z_ * G[7] - 2.0f * y_ * G[8]);
        gq[3] = 2.0f * (-2.0f * z_ * G[0] - w_ * G[1] + x_ * G[2] + w_ * G[3] - 2.0f * z_ * G[4] + y_ * G[5] +
                        x_ * G[6] + y_ * G[7]);
        const float dotq = gq[0] * w_ + gq[1] * x_ + gq[2] * y_ + gq[3] * z_;
        // alpha0 = sigmoid(l)
        const float l = p.logit[n];
        const float a0 = 1.0f / (1.0f + __expf(-l));
        const float glogit = (l < -kLogitMax || l > kLogitMax) ? 0.0f : ga0 * a0 * (1.0f - a0);
        // colour = max(0, 1/2 + sum_k Y_k(d) c_k), d = (mu - campos) / |mu - campos|
        float d[3] = {mu[0] - cam.campos[0], mu[1] - cam.campos[1], mu[2] - cam.campos[2]};
        const float idl = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] *= idl;
        float Y[16], dY[16][3];
        sh_basis_grad<kDeg>(d[0], d[1], d[2], Y, dY);
        float gd[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float pre = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) pre += Y[k] * row[3 * k + ch];
            const float g = pre > 0.0f ? gcol[ch] : 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float cg = row[3 * k + ch] * g;
                gd[0] += cg * dY[k][0];
                gd[1] += cg * dY[k][1];
                gd[2] += cg * dY[k][2];
                row[3 * k + ch] = Y[k] * g;      // the row now holds the SH gradient
            }
        }
        __syncwarp();
        // SH gradient rows out, coalesced
#pragma unroll
        for (int i = 0; i < K3; ++i) {
            const uint32_t idx = (uint32_t)i * 32u + lane, r = idx / K3, k = idx - r * K3;
            const uint32_t nr = __shfl_sync(0xffffffffu, n, r);
            const float g = rows[r * RS + k] + (kAccumulate ? olds[r * RS + k] : 0.0f);
            if (base + r < M) gr.sh[(size_t)nr * K3 + k] = g;
        }
        __syncwarp();
        if (!act) continue;
        const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) gmu[k] += (gd[k] - d[k] * dd) * idl;
        float gqn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) gqn[k] = (gq[k] - qh[k] * dotq) / qn;
        if (kAccumulate) {
            // all eleven loads before the first store (the arrays may alias as far
            // as the compiler knows)
            float o_mu[3], o_ls[3], o_q[4];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o_mu[k] = gr.mu[k * N + n];
                o_ls[k] = gr.log_scale[k * N + n];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) o_q[k] = gr.quat[k * N + n];
            const float o_l = gr.logit[n];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gr.mu[k * N + n] = o_mu[k] + gmu[k];
                gr.log_scale[k * N + n] = o_ls[k] + gls[k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) gr.quat[k * N + n] = o_q[k] + gqn[k];
            gr.logit[n] = o_l + glogit;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gr.mu[k * N + n] = gmu[k];
                gr.log_scale[k * N + n] = gls[k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) gr.quat[k * N + n] = gqn[k];
            gr.logit[n] = glogit;
        }
    }
}

__global__ void __launch_bounds__(128) zero_rows_kernel(float4* __restrict__ gsplat, const FrameState* st)
{
    const uint32_t n4 = st->M * (uint32_t)(kGS / 4);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x)
        gsplat[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_prep_params(const DevTree& t, const float* mu, const float* log_scale, const float* quat,
                        const float* logit, const float* sh, int blocks, cudaStream_t s)
{
    ParamPtrs p{mu, log_scale, quat, logit, sh, t.n};
    prep_params_kernel<<<blocks, 256, 0, s>>>(t, p);
    switch (t.sh_degree) {
    case 0: prep_sh_kernel<0><<<blocks, 256, 0, s>>>(t, sh); break;
    case 1: prep_sh_kernel<1><<<blocks, 256, 0, s>>>(t, sh); break;
    case 2: prep_sh_kernel<2><<<blocks, 256, 0, s>>>(t, sh); break;
    default: prep_sh_kernel<3><<<blocks, 256, 0, s>>>(t, sh); break;
    }
}

template <int kDeg>
static void launch_project_bwd(const DevTree& t, const DevCamera& cam, const ParamPtrs& p,
                               const uint32_t* sel, const float* gsplat, const GradPtrs& gr,
                               bool accumulate, int blocks, FrameState* st, cudaStream_t s)
{
    if (accumulate)
        project_bwd_kernel<kDeg, true><<<blocks, kPbWarps * 32, 0, s>>>(t, cam, p, sel, gsplat, gr, st);
    else
        project_bwd_kernel<kDeg, false><<<blocks, kPbWarps * 32, 0, s>>>(t, cam, p, sel, gsplat, gr, st);
}

void launch_backward(const DevTree& t, const DevCamera& cam, const uint2* ranges, const uint32_t* vals,
                     const float* splat, uint2* keep, bool kept, const uint32_t* sel, const float* dL_drgb,
                     float* gsplat, const float* const params[5], float* const grads[5], bool accumulate,
                     int sms, FrameState* st, cudaStream_t s)
{
    // gsplat rows of the selected Gaussians start at zero: the blend backward adds into them
    zero_rows_kernel<<<sms * 8, 128, 0, s>>>(reinterpret_cast<float4*>(gsplat), st);
    if (kept)
        blend_bwd_kernel<true><<<cam.tiles_x * cam.tiles_y, 256, 0, s>>>(cam, ranges, vals, splat, keep, dL_drgb,
                                                                     gsplat, st);
    else
        blend_bwd_kernel<false><<<cam.tiles_x * cam.tiles_y, 256, 0, s>>>(cam, ranges, vals, splat, keep,
                                                                      dL_drgb, gsplat, st);
    const ParamPtrs p{params[0], params[1], params[2], params[3], params[4], t.n};
    const GradPtrs gr{grads[0], grads[1], grads[2], grads[3], grads[4]};
    if (!accumulate) {
        // nodes outside the selection get zero gradient
        const size_t K3 = (size_t)(t.sh_degree + 1) * (t.sh_degree + 1) * 3;
        cudaMemsetAsync(gr.mu, 0, sizeof(float) * 3 * t.n, s);
        cudaMemsetAsync(gr.log_scale, 0, sizeof(float) * 3 * t.n, s);
        cudaMemsetAsync(gr.quat, 0, sizeof(float) * 4 * t.n, s);
        cudaMemsetAsync(gr.logit, 0, sizeof(float) * t.n, s);
        cudaMemsetAsync(gr.sh, 0, sizeof(float) * K3 * t.n, s);
    }
    const int blocks = sms * (16 / kPbWarps);
    switch (t.sh_degree) {
    case 0: launch_project_bwd<0>(t, cam, p, sel, gsplat, gr, accumulate, blocks, st, s); break;
    case 1: launch_project_bwd<1>(t, cam, p, sel, gsplat, gr, accumulate, blocks, st, s); break;
    case 2: launch_project_bwd<2>(t, cam, p, sel, gsplat, gr, accumulate, blocks, st, s); break;
    default: launch_project_bwd<3>(t, cam, p, sel, gsplat, gr, accumulate, blocks, st, s); break;
    }
}

}  // namespace fgs
