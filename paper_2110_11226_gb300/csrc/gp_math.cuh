// gp_math.cuh -- sin, cos, tan, log and exp for the evaluator's hot loop.
//
// Small inline fast path, out-of-line fallback: the trigonometric fast
// path covers finite |x| < 65536 with a Cody-Waite reduction (W. J. Cody
// and W. Waite, "Software Manual for the Elementary Functions", 1980)
// carried out with three fused multiply-adds against a three-part split of
// the period, then minimax polynomials whose coefficients fit_trig.py
// derives (Lawson's iteration).  sin and cos reduce by pi (cos by an offset
// of half a period) to one odd polynomial on [-pi/2, pi/2]: 1.76 ulp for
// sin and 1.81 ulp for cos over |x| < 65536 (CUDA documents 2 ulp for its
// sinf and cosf).  tan reduces by pi/2 and divides two polynomials on
// [-pi/4, pi/4].  Everything else -- huge arguments, inf, NaN -- goes to
// CUDA's sinf/cosf/tanf through a non-inlined call, so the interpreter's
// inline code stays small.
//
// log: x = 2^k m with m in [sqrt(1/2), sqrt(2)), log x = k ln2 + log(1 + f)
// with f = m - 1 and a degree-9 polynomial for log(1 + f) (coefficients
// from fit_log.py: 1.14 ulp over [0.001, 3.4e38]); it runs on
// max(|a|, 0.001), so no zero, negative or subnormal argument reaches it.
// exp: for |x| < 87, 2^j e^r with j the integer nearest x log2(e), the
// Cody-Waite reduction r = x - j ln2 in two FMAs and a degree-6 polynomial
// (coefficients from fit_exp.py: 1.04 ulp); beyond |x| = 87 the same
// steps scale by 2^j in two exact halves (exp_wide), x >= 89 gives +inf
// and x <= -110 gives +0.  The inline-PTX loop of the evaluator
// transcribes the same steps and constants, so both give the same bits.
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

// pi = HI + MID + LO, and 1/pi rounded
constexpr float kPiHi = 3.1415927410125732f;
constexpr float kPiMid = -8.742277657347586e-08f;
constexpr float kPiLo = -3.4302490200117637e-15f;
constexpr float kInvPi = 0.31830987334251404f;
// sin r ~ r + r^3 (Q0 + r^2 (Q1 + r^2 (Q2 + r^2 Q3))) on [-pi/2, pi/2]
constexpr float kQ0 = -0.16666659712791443f, kQ1 = 0.008333065547049046f,
                kQ2 = -0.0001980953966267407f, kQ3 = 2.6056311526190257e-06f;
// tan's polynomials on [-pi/4, pi/4]:
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
static_assert(__builtin_bit_cast(uint32_t, kPiHi) == 0x40490FDBu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kPiMid) == 0xB3BBBD2Eu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kPiLo) == 0xA7772CEDu, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kInvPi) == 0x3EA2F983u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kQ0) == 0xBE2AAAA6u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kQ1) == 0x3C088769u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kQ2) == 0xB94FB7D4u, "trig constant");
static_assert(__builtin_bit_cast(uint32_t, kQ3) == 0x362EDC67u, "trig constant");
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
// log: the bit pattern of sqrt(1/2) splits x into 2^k m; log(1 + f) ~
// f + f^2 (P0 + f (P1 + ... + f P7)); ln2 = LN2_HI (16 significant bits,
// so k * LN2_HI is exact) + LN2_LO
constexpr uint32_t kSqrtHalfBits = 0x3F3504F3u;
constexpr float kLogP0 = -0.49999991059303284f, kLogP1 = 0.33333951234817505f,
                kLogP2 = -0.25001755356788635f, kLogP3 = 0.19962072372436523f,
                kLogP4 = -0.16570508480072021f, kLogP5 = 0.14917974174022675f,
                kLogP6 = -0.14307521283626556f, kLogP7 = 0.08734840899705887f;
constexpr float kLn2Hi = 0.693145751953125f, kLn2Lo = 1.428606765330187e-06f;
// exp: e^r ~ 1 + r (E1 + r (E2 + ... + r E6)) on |r| <= 0.35
constexpr float kExpE1 = 1.0f, kExpE2 = 0.4999999403953552f, kExpE3 = 0.1666642129421234f,
                kExpE4 = 0.041668057441711426f, kExpE5 = 0.008374955505132675f,
                kExpE6 = 0.001384272240102291f;
constexpr float kLog2e = 1.4426950216293335f;
constexpr float kExpFast = 87.0f;
constexpr float kExpInf = 89.0f, kExpZero = -110.0f;  // e^x is +inf / +0 beyond
static_assert(__builtin_bit_cast(uint32_t, kLogP0) == 0xBEFFFFFDu, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP1) == 0x3EAAAB7Au, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP2) == 0xBE80024Du, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP3) == 0x3E4C6960u, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP4) == 0xBE29AE98u, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP5) == 0x3E18C293u, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP6) == 0xBE12824Fu, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLogP7) == 0x3DB2E3B9u, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLn2Hi) == 0x3F317200u, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kLn2Lo) == 0x35BFBE8Eu, "log constant");
static_assert(__builtin_bit_cast(uint32_t, kExpE1) == 0x3F800000u, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpE2) == 0x3EFFFFFEu, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpE3) == 0x3E2AAA06u, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpE4) == 0x3D2AAC20u, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpE5) == 0x3C09371Cu, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpE6) == 0x3AB57078u, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kLog2e) == 0x3FB8AA3Bu, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpFast) == 0x42AE0000u, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpInf) == 0x42B20000u, "exp constant");
static_assert(__builtin_bit_cast(uint32_t, kExpZero) == 0xC2DC0000u, "exp constant");

// log x for x >= 0.001 (finite; the caller selects inf and NaN itself)
__device__ __forceinline__ float log_pos(float x) {
    const int32_t i = __float_as_int(x);
    const int32_t k = (int32_t)((uint32_t)i - kSqrtHalfBits) >> 23;
    const float m = __int_as_float(i - (int32_t)((uint32_t)k << 23));
    const float f = __fsub_rn(m, 1.0f);
    const float kf = __fsub_rn(__int_as_float(k + 0x4B400000), kRoundMagic);  // exactly k
    float p = __fmaf_rn(kLogP7, f, kLogP6);
    p = __fmaf_rn(p, f, kLogP5);
    p = __fmaf_rn(p, f, kLogP4);
    p = __fmaf_rn(p, f, kLogP3);
    p = __fmaf_rn(p, f, kLogP2);
    p = __fmaf_rn(p, f, kLogP1);
    p = __fmaf_rn(p, f, kLogP0);
    float r = __fmaf_rn(__fmul_rn(f, f), p, f);
    r = __fmaf_rn(kf, kLn2Lo, r);
    return __fmaf_rn(kf, kLn2Hi, r);
}

// e^x for |x| < 87: the product of the polynomial and 2^j is one rounding
__device__ __forceinline__ float exp_fast(float x) {
    const float jm = __fmaf_rn(x, kLog2e, kRoundMagic);
    const float jf = __fsub_rn(jm, kRoundMagic);
    float r = __fmaf_rn(jf, -kLn2Hi, x);
    r = __fmaf_rn(jf, -kLn2Lo, r);
    float p = __fmaf_rn(kExpE6, r, kExpE5);
    p = __fmaf_rn(p, r, kExpE4);
    p = __fmaf_rn(p, r, kExpE3);
    p = __fmaf_rn(p, r, kExpE2);
    p = __fmaf_rn(p, r, kExpE1);
    p = __fmaf_rn(p, r, 1.0f);
    const float s = __int_as_float((int32_t)(((uint32_t)__float_as_int(jm) << 23) + 0x3F800000u));
    return __fmul_rn(p, s);
}

// e^x over the whole float range: exp_fast's steps with 2^j applied as two
// exact powers of two (2^(j >> 1), then the rest), so a product beyond the
// normal range rounds once, to a subnormal or to inf; the same bits as
// exp_fast where |x| < 87.  For -110 < x < 89 (j in [-159, 129], both
// factors normal); NaN gives NaN.
__device__ __forceinline__ float exp_wide(float x) {
    const float jm = __fmaf_rn(x, kLog2e, kRoundMagic);
    const float jf = __fsub_rn(jm, kRoundMagic);
    float r = __fmaf_rn(jf, -kLn2Hi, x);
    r = __fmaf_rn(jf, -kLn2Lo, r);
    float p = __fmaf_rn(kExpE6, r, kExpE5);
    p = __fmaf_rn(p, r, kExpE4);
    p = __fmaf_rn(p, r, kExpE3);
    p = __fmaf_rn(p, r, kExpE2);
    p = __fmaf_rn(p, r, kExpE1);
    p = __fmaf_rn(p, r, 1.0f);
    const int32_t j = __float_as_int(jm) - __float_as_int(kRoundMagic);
    const int32_t ja = j >> 1, jb = j - ja;
    return __fmul_rn(__fmul_rn(p, __int_as_float((ja + 127) << 23)),
                     __int_as_float((jb + 127) << 23));
}

// sin (kind 0) or cos (kind 1) of |x| < 65536: j = the integer nearest
// x/pi - kind/2, r = x - (j + kind/2) pi in [-pi/2, pi/2] (plus rounding
// slack), and the result is sin r, negated when j + kind is odd
__device__ __forceinline__ float sincos_fast(float x, int kind) {
    const float half = kind ? 0.5f : 0.0f;
    const float t1 = __fmaf_rn(x, kInvPi, -half);
    const float jm = __fadd_rn(t1, kRoundMagic);
    const float jh = __fadd_rn(__fsub_rn(jm, kRoundMagic), half);
    float r = __fmaf_rn(jh, -kPiHi, x);
    r = __fmaf_rn(jh, -kPiMid, r);
    r = __fmaf_rn(jh, -kPiLo, r);
    const float s = __fmul_rn(r, r);
    float p = __fmaf_rn(kQ3, s, kQ2);
    p = __fmaf_rn(p, s, kQ1);
    p = __fmaf_rn(p, s, kQ0);
    const float v = __fmaf_rn(p, __fmul_rn(s, r), r);
    return ((__float_as_int(jm) + kind) & 1) ? -v : v;
}

// tan's reduction: r = x - j pi/2, q = j mod 4
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

// Applies sin (kind 0), cos (1) or tan (2) to all RPT rows of a lane:
// the fast paths on every row without branching (so the rows' chains
// interleave), then rows outside the fast path (|x| >= 65536, inf, NaN)
// are redone by CUDA's function behind one test for the whole group.
template <int RPT>
__device__ __forceinline__ void trig_rows(float (&t)[RPT], int kind) {
    float v[RPT];
    bool slow = false;
    if (kind == 2) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            int q;
            const float r = trig_reduce(t[j], q);
            const float s = __fmul_rn(r, r);
            const float sn = sin_poly(r, s), cs = cos_poly(s);
            v[j] = (q & 1) ? -__fdiv_rn(cs, sn) : __fdiv_rn(sn, cs);
            slow |= !(fabsf(t[j]) < kTrigFast);
        }
    } else {
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            v[j] = sincos_fast(t[j], kind);
            slow |= !(fabsf(t[j]) < kTrigFast);
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
