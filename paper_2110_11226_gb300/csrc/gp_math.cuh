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

// the extended function set: two rounded products, CUDA's float functions,
// and max / min with NaN from either operand and the right operand on ties
__device__ __forceinline__ float f_sq(float a) { return __fmul_rn(a, a); }
__device__ __forceinline__ float f_cube(float a) { return __fmul_rn(__fmul_rn(a, a), a); }
__device__ __forceinline__ float f_cbrt(float a) { return cbrtf(a); }
__device__ __forceinline__ float f_tanh(float a) { return tanhf(a); }
__device__ __forceinline__ float f_atan(float a) { return atanf(a); }
__device__ __forceinline__ float f_sinh(float a) { return sinhf(a); }
__device__ __forceinline__ float f_cosh(float a) { return coshf(a); }
__device__ __forceinline__ float f_max(float a, float b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ float f_min(float a, float b) { return (a < b || a != a) ? a : b; }

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

// r = x - j pi/2 with j the integer nearest x 2/pi, q = j mod 4.  Adding
// 1.5 * 2^23 rounds to an integer in the FMA pipe, and for |j| < 2^22 the
// two's-complement low bits of that sum's encoding are j's low bits.
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23

// The evaluator's fast loop (inline PTX) spells these constants as float
// bit patterns; the checks keep the two spellings the same numbers.
static_assert(__builtin_bit_cast(uint32_t, kPio2Hi) == 0x3FC90FDBu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kPio2Mid) == 0xB33BBD2Eu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kPio2Lo) == 0xA6F72CEDu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kTwoOverPi) == 0x3F22F983u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kS0) == 0xBE2AAAABu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kS1) == 0x3C088884u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kS2) == 0xB95007C0u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kS3) == 0x363668F9u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kC0) == 0x3D2AAAABu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kC1) == 0xBAB60B5Cu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kC2) == 0x37D0086Fu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kC3) == 0xB4920F4Eu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kRoundMagic) == 0x4B400000u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kTrigFast) == 0x47800000u, "trig constant");
__device__ __forceinline__ float trig_reduce(float x, int &q) {
    const float jm = __fmaf_rn(x, kTwoOverPi, kRoundMagic);
    const float j = __fsub_rn(jm, kRoundMagic);
    q = __float_as_int(jm);
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

static __device__ __noinline__ float trig_slow(float x, int kind) {
    return kind == 0 ? sinf(x) : (kind == 1 ? cosf(x) : tanf(x));
}

// Applies sin (kind 0), cos (1) or tan (2) to all RPT rows of a lane with
// one body for the three: reduction and both polynomials on every row
// without branching (so the rows' chains interleave), then the quadrant
// select (sin, cos) or the quotient (tan); rows outside the fast path
// (|x| >= 65536, inf, NaN) are redone by CUDA's function behind one test
// for the whole group.
template <int RPT>
__device__ __forceinline__ void trig_rows(float (&t)[RPT], int kind) {
    float sn[RPT], cs[RPT];
    int q[RPT];
    bool slow = false;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const float r = trig_reduce(t[j], q[j]);
        const float s = __fmul_rn(r, r);
        sn[j] = sin_poly(r, s);
        cs[j] = cos_poly(s);
        slow |= !(fabsf(t[j]) < kTrigFast);
    }
    float v[RPT];
    if (kind == 2) {
#pragma unroll
        for (int j = 0; j < RPT; ++j)
            v[j] = (q[j] & 1) ? -__fdiv_rn(cs[j], sn[j]) : __fdiv_rn(sn[j], cs[j]);
    } else {
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int qq = q[j] + kind;
            const float a = (qq & 1) ? cs[j] : sn[j];
            v[j] = (qq & 2) ? -a : a;
        }
    }
    if (slow) {
#pragma unroll
        for (int j = 0; j < RPT; ++j)
            if (!(fabsf(t[j]) < kTrigFast)) v[j] = trig_slow(t[j], kind);
    }
#pragma unroll
    for (int j = 0; j < RPT; ++j) t[j] = v[j];
}

}  // namespace gpk
