// gp_math.cuh -- sin, cos and tan for the evaluator's hot loop.
//
// Small inline fast path, out-of-line fallback: the fast path covers finite
// |x| < 65536 with a Cody-Waite reduction by pi/2 (W. J. Cody and W. Waite,
// "Software Manual for the Elementary Functions", 1980) carried out with
// three fused multiply-adds against a three-part split of pi/2, then
// polynomials on [-pi/4, pi/4] whose coefficients fit_trig.py derives (a
// minimax fit by Lawson's iteration, < 1 ulp in float32 on the interval).
// Everything else -- huge arguments, inf, NaN -- goes to CUDA's sinf/cosf
// through a non-inlined call, so the interpreter's inline code stays small.
#pragma once

#include <cstdint>

namespace gpk {

constexpr float kTrigFast = 65536.0f;

// pi/2 = HI + MID + LO (float32 parts of the exact value)
constexpr float kPio2Hi = 1.57079637f;
constexpr float kPio2Mid = -4.37113883e-08f;
constexpr float kPio2Lo = -1.71512451e-15f;
constexpr float kTwoOverPi = 0.636619747f;

// sin r ~ r + r^3 (S0 + r^2 (S1 + r^2 (S2 + r^2 S3)))
constexpr float kS0 = -0.166666672f, kS1 = 0.00833332911f, kS2 = -0.000198393129f,
                kS3 = 2.71812155e-06f;
// cos r ~ 1 + r^2 (-1/2 + r^2 (C0 + r^2 (C1 + r^2 (C2 + r^2 C3))))
constexpr float kC0 = 0.0416666679f, kC1 = -0.00138888834f, kC2 = 2.47994594e-05f,
                kC3 = -2.72057548e-07f;

static __device__ __noinline__ float gp_sin_slow(float x) { return sinf(x); }
static __device__ __noinline__ float gp_cos_slow(float x) { return cosf(x); }
static __device__ __noinline__ float gp_tan_slow(float x) { return tanf(x); }

// r = x - j pi/2 with j = rint(x 2/pi); q = j
__device__ __forceinline__ float trig_reduce(float x, int &q) {
    const float j = rintf(__fmul_rn(x, kTwoOverPi));
    q = (int)j;
    float r = __fmaf_rn(-j, kPio2Hi, x);
    r = __fmaf_rn(-j, kPio2Mid, r);
    r = __fmaf_rn(-j, kPio2Lo, r);
    return r;
}

__device__ __forceinline__ float sin_poly(float r, float s) {
    float p = __fmaf_rn(kS3, s, kS2);
    p = __fmaf_rn(p, s, kS1);
    p = __fmaf_rn(p, s, kS0);
    return __fmaf_rn(p, __fmul_rn(s, r), r);
}

__device__ __forceinline__ float cos_poly(float s) {
    float p = __fmaf_rn(kC3, s, kC2);
    p = __fmaf_rn(p, s, kC1);
    p = __fmaf_rn(p, s, kC0);
    p = __fmaf_rn(p, s, -0.5f);
    return __fmaf_rn(p, s, 1.0f);
}

// quadrant q (mod 4) of x = q pi/2 + r: sin x = sin r, cos r, -sin r, -cos r
__device__ __forceinline__ float gp_sin(float x) {
    if (!(fabsf(x) < kTrigFast)) return gp_sin_slow(x);
    int q;
    const float r = trig_reduce(x, q);
    const float s = __fmul_rn(r, r);
    const float v = (q & 1) ? cos_poly(s) : sin_poly(r, s);
    return (q & 2) ? -v : v;
}

__device__ __forceinline__ float gp_cos(float x) {
    if (!(fabsf(x) < kTrigFast)) return gp_cos_slow(x);
    int q;
    const float r = trig_reduce(x, q);
    const float s = __fmul_rn(r, r);
    q += 1;
    const float v = (q & 1) ? cos_poly(s) : sin_poly(r, s);
    return (q & 2) ? -v : v;
}

// tan x = sin r / cos r (q even) or -cos r / sin r (q odd)
__device__ __forceinline__ float gp_tan(float x) {
    if (!(fabsf(x) < kTrigFast)) return gp_tan_slow(x);
    int q;
    const float r = trig_reduce(x, q);
    const float s = __fmul_rn(r, r);
    const float sn = sin_poly(r, s), cs = cos_poly(s);
    return (q & 1) ? -__fdiv_rn(cs, sn) : __fdiv_rn(sn, cs);
}

}  // namespace gpk
