// Per-Gaussian projection shared by the single-view and the batched kernels:
// EWA projection, footprint (3 sigma or shrunk to tau, §3.3), tile rectangle,
// pair count and SH colour.  Decision quantities use the explicitly rounded
// binary32 helpers of fgs_internal.cuh.
#pragma once

#include "fgs_internal.cuh"

namespace fgs {
namespace proj {


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


// Project node n (selected rank m) with camera cam: writes the 48-byte splat
// record splat[m] and the footprint record foot[m] = {x0 | x1 << 16,
// y0 | y1 << 16, pair count, depth bits}, and returns the footprint record.
__device__ __forceinline__ uint4 project_one(const DevTree& t, const DevCamera& cam, uint32_t n,
                                                uint32_t m, float* __restrict__ splat,
                                                uint4* __restrict__ foot)
{
    const float ftx = (float)cam.tiles_x, fty = (float)cam.tiles_y;
    uint32_t cnt = 0;
    // ---- decision-exact binary32: frustum, EWA covariance, footprint
    const float4 q0 = __ldg(t.attr + 3 * (size_t)n);
    const float4 q1 = __ldg(t.attr + 3 * (size_t)n + 1);
    const float4 q2 = __ldg(t.attr + 3 * (size_t)n + 2);
    const float mx = q0.x, my = q0.y, mz = q0.z;
    const float s6[6] = {q1.x, q1.y, q1.z, q1.w, q2.x, q2.y};
    const float a0 = q0.w;
    const float ln_a0 = q2.z;
    float vx, vy, vz, txtz = 0.0f, tytz = 0.0f;
    camera_space(cam, mx, my, mz, vx, vy, vz);
    const bool inf = frustum_test(cam, vx, vy, vz, txtz, tytz);
    float a = 0.0f, b = 0.0f, c = 0.0f, lam = 0.0f;
    if (inf) ewa_cov2d(cam, vz, txtz, tytz, s6, a, b, c, lam);
    // x / z and y / z: the frustum test's quotients when it formed them (depth above 0.2)
    const float u = fa(fm(cam.fx, vz > 0.2f ? txtz : fd(vx, vz)), cam.cx);
    const float v = fa(fm(cam.fy, vz > 0.2f ? tytz : fd(vy, vz)), cam.cy);
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
            // tiles are powers of two wide and high, so x / w is x * (1 / w) bit for bit
            // (both the correctly rounded x * 2^-k)
            const float iw = __uint_as_float((uint32_t)(127 - cam.tile_shift_x) << 23);
            const float ih = __uint_as_float((uint32_t)(127 - cam.tile_shift_y) << 23);
            const float fx0 = clampf(floorf(fm(fs(u, r), iw)), 0.0f, ftx);
            const float fx1 = clampf(fa(floorf(fm(fa(u, r), iw)), 1.0f), 0.0f, ftx);
            const float fy0 = clampf(floorf(fm(fs(v, r), ih)), 0.0f, fty);
            const float fy1 = clampf(fa(floorf(fm(fa(v, r), ih)), 1.0f), 0.0f, fty);
            x0 = (int32_t)fx0; x1 = (int32_t)fx1; y0 = (int32_t)fy0; y1 = (int32_t)fy1;
            if (x1 > x0 && y1 > y0) cnt = (uint32_t)((x1 - x0) * (y1 - y0));
        }
    }
    const uint4 fr = make_uint4((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16),
                                cnt, __float_as_uint(vz));
    foot[m] = fr;
    // ---- colour (FMA allowed: decides nothing), only for a Gaussian that emits
    // pairs: no pixel ever reads the colour of one that does not (about 40% of
    // the selection under shrinking), so its SH row is not fetched
    float rgb[3] = {0.0f, 0.0f, 0.0f};
    if (cnt) {
        float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= il; dy *= il; dz *= il;
        sh_colour(t.sh + (size_t)n * t.sh_stride, (int)t.sh_degree, dx, dy, dz, rgb);
    }
    float4* out = reinterpret_cast<float4*>(splat + (size_t)m * kSplatStride);
    out[0] = make_float4(u, v, A, B);
    out[1] = make_float4(C, lthr, a0, vz);
    out[2] = make_float4(rgb[0], rgb[1], rgb[2], radius);
    return fr;
}

}  // namespace proj
}  // namespace fgs
