// gp_interp.cuh -- the batched persistent evaluator (the hot loop).
//
// Work: every (program, row-chunk) pair of one program class is an item of a
// dynamic queue (one atomic counter); items are ordered chunk-major and,
// inside a chunk, longest program first, so the blocks that share the GPU
// at any moment work on the same few row chunks (X stays in L2) and the
// queue drains with the short items last.
//
// A block takes one item, the way the paper's execution kernel gives each
// block one program (Sec. III-C3, III-D1): the program's compiled
// instructions are copied once into shared memory and every warp of the
// block runs that same instruction stream over its own sub-tiles of 32*RPT
// rows (sub-tile w, w + warps, ...).  Within a warp the instruction stream
// is uniform, so the dispatch switch never diverges; across the block the
// warps walk the same few switch cases, which keeps the SM's instruction
// working set small.  Lane l owns rows base + l*RPT .. +RPT-1 (vectorised,
// coalesced loads from the column-major X).  The top of the stack is the
// register array t[RPT]; deeper values sit in the warp's slice of a
// shared-memory stack, one float4 per (slot, group of 4 rows, lane), so a
// push or pop is one or two conflict-free 16-byte accesses per lane.  Each
// instruction costs one indexed branch (the inline-PTX fast loop, 4 rows per
// lane) or one switch, and nothing else that branches:
// measured on this GPU, an interpreter's dispatch latency grows with every
// dependent branch per instruction (about 20-40 cycles each) and with the
// number of distinct code locations it jumps between, so operand source and
// spill are part of the operation code rather than separate tests.
//
// After a sub-tile each lane turns its RPT predictions into weighted losses
// (the fused form of the paper's matrix-vector loss step) and adds them into
// a Kahan-compensated FP32 sum; at the end of the item each warp adds its 32
// lane sums with a fixed butterfly and thread 0 adds the warp sums in warp
// order, writing one partial per (program, chunk).  A separate pass adds the
// partials of a program in chunk order in FP64.  Every step has a fixed
// order, so results do not depend on which block ran which item.
#pragma once

#include "gp_internal.cuh"
#include "gp_math.cuh"

namespace gpk {

// warps per block: 8, or 4 at 16 rows per thread (its shared-memory stack
// is twice as large per warp)
template <int RPT>
__host__ __device__ constexpr int eval_warps() { return RPT >= 16 ? 4 : 8; }

// ---- the function set (FP32, IEEE operators, no contraction) -----------
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
// The protected operators compute the operation on every row and select
// afterwards: written as a branch around the operation, the compiler keeps
// a per-row branch, which costs more than the operation saved (measured).
__device__ __forceinline__ float f_div(float a, float b) {
    const float q = __fdiv_rn(a, b);
    return fabsf(b) < kThr ? 1.0f : q;
}
__device__ __forceinline__ float f_sqrt(float a) { return __fsqrt_rn(fabsf(a)); }
__device__ __forceinline__ float f_log(float a) {
    // logf sees an argument >= thr, which spares it its tiny-argument
    // paths; NaN, for which both tests fail, is passed through
    const float b = fabsf(a);
    const float l = logf(fmaxf(b, kThr));
    return b >= kThr ? l : (b < kThr ? 0.0f : b);
}
__device__ __forceinline__ float f_exp(float a) { return expf(a); }
__device__ __forceinline__ float f_abs(float a) { return fabsf(a); }
__device__ __forceinline__ float f_neg(float a) { return -a; }
__device__ __forceinline__ float f_inv(float a) {
    const float r = __frcp_rn(a);
    return fabsf(a) < kThr ? 0.0f : r;
}

// per-row loss (metric readings of Sec. III-C3, FP32)
__device__ __forceinline__ float row_loss(int metric, float p, float y) {
    if (metric == GP_MAE) return fabsf(__fsub_rn(p, y));
    if (metric == GP_LOGLOSS) {
        const float ap = fabsf(p);
        const float c = (p >= 0.0f) ? __fsub_rn(1.0f, y) : y;
        const float lin = (c == 0.0f) ? 0.0f : __fmul_rn(c, ap);
        return __fadd_rn(lin, log1pf(expf(-ap)));
    }
    const float d = __fsub_rn(p, y);
    return __fmul_rn(d, d);
}

// RPT consecutive rows starting at r0 of one column; rows >= re read 0.
template <int RPT>
__device__ __forceinline__ void load_rows(float (&v)[RPT], const float *__restrict__ col,
                                          int64_t r0, int64_t re, bool vec) {
    if (vec && r0 + RPT <= re) {
#pragma unroll
        for (int q = 0; q < RPT / 4; ++q) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(col + r0) + q);
            v[4 * q + 0] = f.x;
            v[4 * q + 1] = f.y;
            v[4 * q + 2] = f.z;
            v[4 * q + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < RPT; ++j) v[j] = (r0 + j < re) ? __ldg(col + r0 + j) : 0.0f;
    }
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float yv = __fsub_rn(x, c);
    const float tv = __fadd_rn(s, yv);
    // once the sum is infinite or NaN the compensation is meaningless
    c = isfinite(tv) ? __fsub_rn(__fsub_rn(tv, s), yv) : 0.0f;
    s = tv;
}

// The extended unary functions of four rows, out of line: with a case of
// their own each in the dispatch switch (a 6-bit switch), their code made
// the loop 4-5% slower on programs that never use them (measured on
// Pagie-1 x 4096 programs).
static __device__ __noinline__ float4 ext_rows4(float4 v, uint32_t f) {
    switch (f) {
        case EXT_SQ: return make_float4(f_sq(v.x), f_sq(v.y), f_sq(v.z), f_sq(v.w));
        case EXT_CUBE: return make_float4(f_cube(v.x), f_cube(v.y), f_cube(v.z), f_cube(v.w));
        case EXT_CBRT: return make_float4(f_cbrt(v.x), f_cbrt(v.y), f_cbrt(v.z), f_cbrt(v.w));
        case EXT_TANH: return make_float4(f_tanh(v.x), f_tanh(v.y), f_tanh(v.z), f_tanh(v.w));
        case EXT_ATAN: return make_float4(f_atan(v.x), f_atan(v.y), f_atan(v.z), f_atan(v.w));
        case EXT_SINH: return make_float4(f_sinh(v.x), f_sinh(v.y), f_sinh(v.z), f_sinh(v.w));
        default: return make_float4(f_cosh(v.x), f_cosh(v.y), f_cosh(v.z), f_cosh(v.w));
    }
}

// ---- the fast loop: indexed-branch dispatch in inline PTX ------------
// The compiler lowers the dispatch switch to a tree of compares and
// branches (about 12 instructions per dispatch, measured with ncu's
// per-opcode counts); PTX's brx.idx jumps through a table instead (about
// 3).  This loop, 4 rows per lane, runs the operations whose evaluator
// semantics PTX states directly:
//   * pushes and stack moves, abs and neg, and IEEE adds, subtracts and
//     multiplies with every operand form (add/sub/mul.rn.f32, the
//     instructions behind __fadd_rn, __fsub_rn and __fmul_rn);
//   * column reads when columns 0 and 1 are held in registers (XREG);
//   * with DIVS, the protected divisions, square root and reciprocal
//     (div/sqrt/rcp.rn.f32, as __fdiv_rn, __fsqrt_rn and __frcp_rn, all
//     without flush to zero, then the protection selects) and sin, cos and
//     tan (the steps and constants of trig_rows, transcribed).
// It stops at the first word it does not run (OP_END, log, exp, the
// extended functions, trigonometric arguments outside the fast path, and
// whatever XREG or DIVS leave out), hands that word and its constant back
// to the caller's switch and leaves pa just past it.  Every one of the 32
// values of the 5-bit op field has a table entry, so the index is always
// in range; stack slots are clamped like the switch's.
// Measured on Pagie-1 16M x 4096: 465 ms -> 420 ms per evaluation, 390 ms
// with the trigonometry; the 28-column table, its column reads handed
// back, 119 ms -> 112 ms.  DIVS is off in the instances with the extended
// functions: there it cost the extended-set population 23% (their
// out-of-line calls and the division's own slow-path call do not mix
// well).  Loading the next word while the current one runs cost 3%.
//
// the op tables: with DIVS the division set (7 DIV_S .. 19 RDIV_C, 20 SQRT,
// 28 INV) and trigonometry (23 SIN .. 25 TAN) run here, otherwise they are
// handed back
#define GP_FAST_TABLE_DIVS                                                        \
    "T%=: .branchtargets PX%=, PC%=, PXS%=, PCS%=, AS%=, SS%=, MS%=, DS%=,"       \
    " AX%=, AC%=, SX%=, SC%=, RX%=, RC%=, MX%=, MC%=, DX%=, DC%=, RDX%=, RDC%=,"  \
    " SQ%=, EX%=, EX%=, TSC%=, TSC%=, TTN%=, AB%=, NG%=, IV%=, EX%=, EX%=, EX%=;\n\t"
#define GP_FAST_TABLE_NODIVS                                                      \
    "T%=: .branchtargets PX%=, PC%=, PXS%=, PCS%=, AS%=, SS%=, MS%=, EX%=,"       \
    " AX%=, AC%=, SX%=, SC%=, RX%=, RC%=, MX%=, MC%=, EX%=, EX%=, EX%=, EX%=,"    \
    " EX%=, EX%=, EX%=, EX%=, EX%=, EX%=, AB%=, NG%=, EX%=, EX%=, EX%=, EX%=;\n\t"
// without columns in registers (more than 2 features) the column reads
// (PUSH_X, PUSH_X_SP and the _X forms) are handed back too
#define GP_FAST_TABLE_DIVS_NOX                                                    \
    "T%=: .branchtargets EX%=, PC%=, EX%=, PCS%=, AS%=, SS%=, MS%=, DS%=,"        \
    " EX%=, AC%=, EX%=, SC%=, EX%=, RC%=, EX%=, MC%=, EX%=, DC%=, EX%=, RDC%=,"   \
    " SQ%=, EX%=, EX%=, TSC%=, TSC%=, TTN%=, AB%=, NG%=, IV%=, EX%=, EX%=, EX%=;\n\t"
#define GP_FAST_TABLE_NODIVS_NOX                                                  \
    "T%=: .branchtargets EX%=, PC%=, EX%=, PCS%=, AS%=, SS%=, MS%=, EX%=,"        \
    " EX%=, AC%=, EX%=, SC%=, EX%=, RC%=, EX%=, MC%=, EX%=, EX%=, EX%=, EX%=,"    \
    " EX%=, EX%=, EX%=, EX%=, EX%=, EX%=, AB%=, NG%=, EX%=, EX%=, EX%=, EX%=;\n\t"
#define GP_FAST_LOOP_TOP                                                          \
    "N%=:\n\t"                                                                    \
    "ld.shared.v2.b32 {%%w, %%cb}, [%0];\n\t"                                     \
    "mov.b32 %%cf, %%cb;\n\t"                                                     \
    "add.u32 %0, %0, 8;\n\t"                                                      \
    "and.b32 %%i, %%w, 31;\n\t"                                                   \
    "brx.idx.uni %%i, T%=;\n\t"
#define GP_FAST_HEAD(TABLE)                                                       \
    "{\n\t"                                                                       \
    ".reg .pred %%p;\n\t"                                                         \
    ".reg .b32 %%w, %%cb, %%i, %%a, %%f;\n\t"                                     \
    ".reg .f32 %%cf, %%u0, %%u1, %%u2, %%u3, %%q, %%m;\n\t"                       \
    TABLE GP_FAST_LOOP_TOP
// slot address: sb + min(slot, NSLOT - 1) * 512 (one float4 per lane, 32 lanes)
#define GP_FAST_SLOT                                                              \
    "bfe.u32 %%a, %%w, 8, 8;\n\t"                                                 \
    "min.u32 %%a, %%a, %8;\n\t"                                                   \
    "mad.lo.u32 %%a, %%a, 512, %7;\n\t"
#define GP_FAST_SPILL GP_FAST_SLOT "st.shared.v4.f32 [%%a], {%1, %2, %3, %4};\n\t"
#define GP_FAST_SLOTLOAD GP_FAST_SLOT "ld.shared.v4.f32 {%%u0, %%u1, %%u2, %%u3}, [%%a];\n\t"
// columns 0 and 1 in registers (x1 when the feature is not 0)
#define GP_FAST_X(D0, D1, D2, D3)                                                 \
    "shr.b32 %%f, %%w, 16;\n\t"                                                   \
    "setp.ne.u32 %%p, %%f, 0;\n\t"                                                \
    "selp.f32 " D0 ", %13, %9, %%p;\n\tselp.f32 " D1 ", %14, %10, %%p;\n\t"       \
    "selp.f32 " D2 ", %15, %11, %%p;\n\tselp.f32 " D3 ", %16, %12, %%p;\n\t"
#define GP_FAST_XU GP_FAST_X("%%u0", "%%u1", "%%u2", "%%u3")
// t_j = t_j OP v_j for the four rows (v: "%%u" or the constant "%%cf")
#define GP_FAST_TV(OP, V0, V1, V2, V3)                                            \
    OP ".rn.f32 %1, %1, " V0 ";\n\t" OP ".rn.f32 %2, %2, " V1 ";\n\t"             \
    OP ".rn.f32 %3, %3, " V2 ";\n\t" OP ".rn.f32 %4, %4, " V3 ";\n\t"
#define GP_FAST_TU(OP) GP_FAST_TV(OP, "%%u0", "%%u1", "%%u2", "%%u3")
#define GP_FAST_TC(OP) GP_FAST_TV(OP, "%%cf", "%%cf", "%%cf", "%%cf")
// t_j = v_j - t_j
#define GP_FAST_RSUB(V0, V1, V2, V3)                                              \
    "sub.rn.f32 %1, " V0 ", %1;\n\tsub.rn.f32 %2, " V1 ", %2;\n\t"                \
    "sub.rn.f32 %3, " V2 ", %3;\n\tsub.rn.f32 %4, " V3 ", %4;\n\t"
// protected division of one row: D = |B| < thr ? 1 : A / B
#define GP_FAST_DIV1(D, A, B)                                                     \
    "div.rn.f32 %%q, " A ", " B ";\n\t"                                           \
    "abs.f32 %%m, " B ";\n\t"                                                     \
    "setp.lt.f32 %%p, %%m, %17;\n\t"                                              \
    "selp.f32 " D ", 0f3F800000, %%q, %%p;\n\t"
#define GP_FAST_DIV_TV(V0, V1, V2, V3)                                            \
    GP_FAST_DIV1("%1", "%1", V0) GP_FAST_DIV1("%2", "%2", V1)                     \
    GP_FAST_DIV1("%3", "%3", V2) GP_FAST_DIV1("%4", "%4", V3)
#define GP_FAST_DIV_VT(V0, V1, V2, V3)                                            \
    GP_FAST_DIV1("%1", V0, "%1") GP_FAST_DIV1("%2", V1, "%2")                     \
    GP_FAST_DIV1("%3", V2, "%3") GP_FAST_DIV1("%4", V3, "%4")
#define GP_FAST_SQRT1(T) "abs.f32 " T ", " T ";\n\tsqrt.rn.f32 " T ", " T ";\n\t"
// protected reciprocal: |t| < thr ? 0 : 1 / t
#define GP_FAST_INV1(T)                                                           \
    "rcp.rn.f32 %%q, " T ";\n\t"                                                  \
    "abs.f32 %%m, " T ";\n\t"                                                     \
    "setp.lt.f32 %%p, %%m, %17;\n\t"                                              \
    "selp.f32 " T ", 0f00000000, %%q, %%p;\n\t"
#define GP_FAST_SETC                                                              \
    "mov.f32 %1, %%cf;\n\tmov.f32 %2, %%cf;\n\tmov.f32 %3, %%cf;\n\tmov.f32 %4, %%cf;\n\t"
#define GP_FAST_NEXT "bra.uni N%=;\n\t"
// sin, cos and tan of the four rows with the steps and constants of
// trig_rows (gp_math.cuh): Cody-Waite reduction by pi/2 in three FMAs,
// both polynomials, then the quadrant select or the quotient, so the
// results are the same bits.  A warp with any row outside the fast path
// (|x| >= 65536, inf, NaN) hands the word back before touching t, and the
// caller's switch runs trig_rows with its slow path.
#define GP_FAST_TRIG_REGS                                                         \
    ".reg .pred %%ps;\n\t"                                                        \
    ".reg .b32 %%qq, %%qb, %%kd;\n\t"                                             \
    ".reg .f32 %%jm, %%jj, %%rr, %%ss, %%sn, %%cn, %%sr;\n\t"
#define GP_FAST_TRIG_CHECK1(T)                                                    \
    "abs.f32 %%m, " T ";\n\t"                                                     \
    "setp.geu.f32 %%p, %%m, 0f47800000;\n\t"                                      \
    "or.pred %%ps, %%ps, %%p;\n\t"
#define GP_FAST_TRIG_CHECK                                                        \
    "setp.ne.u32 %%ps, 0, 0;\n\t"                                                 \
    GP_FAST_TRIG_CHECK1("%1") GP_FAST_TRIG_CHECK1("%2")                           \
    GP_FAST_TRIG_CHECK1("%3") GP_FAST_TRIG_CHECK1("%4")                           \
    "vote.sync.any.pred %%ps, %%ps, 0xffffffff;\n\t"                              \
    "@%%ps bra EX%=;\n\t"
// reduction and both polynomials of row T: %%sn = sin r, %%cn = cos r,
// %%qq = the quadrant word (low bits of j)
#define GP_FAST_TRIG_POLY(T)                                                      \
    "fma.rn.f32 %%jm, " T ", 0f3F22F983, 0f4B400000;\n\t"                         \
    "sub.rn.f32 %%jj, %%jm, 0f4B400000;\n\t"                                      \
    "neg.f32 %%jj, %%jj;\n\t"                                                     \
    "fma.rn.f32 %%rr, %%jj, 0f3FC90FDB, " T ";\n\t"                               \
    "fma.rn.f32 %%rr, %%jj, 0fB33BBD2E, %%rr;\n\t"                                \
    "fma.rn.f32 %%rr, %%jj, 0fA6F72CED, %%rr;\n\t"                                \
    "mul.rn.f32 %%ss, %%rr, %%rr;\n\t"                                            \
    "fma.rn.f32 %%sn, 0f363668F9, %%ss, 0fB95007C0;\n\t"                          \
    "fma.rn.f32 %%sn, %%sn, %%ss, 0f3C088884;\n\t"                                \
    "fma.rn.f32 %%sn, %%sn, %%ss, 0fBE2AAAAB;\n\t"                                \
    "mul.rn.f32 %%sr, %%ss, %%rr;\n\t"                                            \
    "fma.rn.f32 %%sn, %%sn, %%sr, %%rr;\n\t"                                      \
    "fma.rn.f32 %%cn, 0fB4920F4E, %%ss, 0f37D0086F;\n\t"                          \
    "fma.rn.f32 %%cn, %%cn, %%ss, 0fBAB60B5C;\n\t"                                \
    "fma.rn.f32 %%cn, %%cn, %%ss, 0f3D2AAAAB;\n\t"                                \
    "fma.rn.f32 %%cn, %%cn, %%ss, 0fBF000000;\n\t"                                \
    "fma.rn.f32 %%cn, %%cn, %%ss, 0f3F800000;\n\t"                                \
    "mov.b32 %%qq, %%jm;\n\t"
// sin (kind 0) or cos (kind 1, in %%kd): a = ((q + kind) & 1) ? cos : sin,
// negated when (q + kind) & 2
#define GP_FAST_SINCOS1(T)                                                        \
    GP_FAST_TRIG_POLY(T)                                                          \
    "add.u32 %%qq, %%qq, %%kd;\n\t"                                               \
    "and.b32 %%qb, %%qq, 1;\n\t"                                                  \
    "setp.ne.u32 %%p, %%qb, 0;\n\t"                                               \
    "selp.f32 %%sn, %%cn, %%sn, %%p;\n\t"                                         \
    "and.b32 %%qb, %%qq, 2;\n\t"                                                  \
    "setp.ne.u32 %%p, %%qb, 0;\n\t"                                               \
    "neg.f32 %%cn, %%sn;\n\t"                                                     \
    "selp.f32 " T ", %%cn, %%sn, %%p;\n\t"
// tan: (q & 1) ? -(cos / sin) : sin / cos
#define GP_FAST_TAN1(T)                                                           \
    GP_FAST_TRIG_POLY(T)                                                          \
    "and.b32 %%qb, %%qq, 1;\n\t"                                                  \
    "setp.ne.u32 %%p, %%qb, 0;\n\t"                                               \
    "selp.f32 %%q, %%cn, %%sn, %%p;\n\t"                                          \
    "selp.f32 %%m, %%sn, %%cn, %%p;\n\t"                                          \
    "div.rn.f32 %%q, %%q, %%m;\n\t"                                               \
    "neg.f32 %%m, %%q;\n\t"                                                       \
    "selp.f32 " T ", %%m, %%q, %%p;\n\t"
#define GP_FAST_TRIG_BODIES                                                       \
    "TSC%=:\n\t" GP_FAST_TRIG_CHECK                                               \
    "sub.u32 %%kd, %%i, 23;\n\t"                                                  \
    GP_FAST_SINCOS1("%1") GP_FAST_SINCOS1("%2") GP_FAST_SINCOS1("%3")             \
    GP_FAST_SINCOS1("%4") GP_FAST_NEXT                                            \
    "TTN%=:\n\t" GP_FAST_TRIG_CHECK                                               \
    GP_FAST_TAN1("%1") GP_FAST_TAN1("%2") GP_FAST_TAN1("%3") GP_FAST_TAN1("%4")   \
    GP_FAST_NEXT
#define GP_FAST_DIV_BODIES                                                        \
    "DS%=:\n\t" GP_FAST_SLOTLOAD GP_FAST_DIV_TV("%%u0", "%%u1", "%%u2", "%%u3") GP_FAST_NEXT \
    "DX%=:\n\t" GP_FAST_XU GP_FAST_DIV_TV("%%u0", "%%u1", "%%u2", "%%u3") GP_FAST_NEXT \
    "DC%=:\n\t" GP_FAST_DIV_TV("%%cf", "%%cf", "%%cf", "%%cf") GP_FAST_NEXT       \
    "RDX%=:\n\t" GP_FAST_XU GP_FAST_DIV_VT("%%u0", "%%u1", "%%u2", "%%u3") GP_FAST_NEXT \
    "RDC%=:\n\t" GP_FAST_DIV_VT("%%cf", "%%cf", "%%cf", "%%cf") GP_FAST_NEXT      \
    "SQ%=:\n\t" GP_FAST_SQRT1("%1") GP_FAST_SQRT1("%2") GP_FAST_SQRT1("%3")       \
    GP_FAST_SQRT1("%4") GP_FAST_NEXT                                              \
    "IV%=:\n\t" GP_FAST_INV1("%1") GP_FAST_INV1("%2") GP_FAST_INV1("%3")          \
    GP_FAST_INV1("%4") GP_FAST_NEXT
#define GP_FAST_BODY                                                              \
    "PX%=:\n\t" GP_FAST_X("%1", "%2", "%3", "%4") GP_FAST_NEXT                    \
    "PC%=:\n\t" GP_FAST_SETC GP_FAST_NEXT                                         \
    "PXS%=:\n\t" GP_FAST_SPILL GP_FAST_X("%1", "%2", "%3", "%4") GP_FAST_NEXT     \
    "PCS%=:\n\t" GP_FAST_SPILL GP_FAST_SETC GP_FAST_NEXT                          \
    "AS%=:\n\t" GP_FAST_SLOTLOAD GP_FAST_TU("add") GP_FAST_NEXT                   \
    "SS%=:\n\t" GP_FAST_SLOTLOAD GP_FAST_TU("sub") GP_FAST_NEXT                   \
    "MS%=:\n\t" GP_FAST_SLOTLOAD GP_FAST_TU("mul") GP_FAST_NEXT                   \
    "AX%=:\n\t" GP_FAST_XU GP_FAST_TU("add") GP_FAST_NEXT                         \
    "AC%=:\n\t" GP_FAST_TC("add") GP_FAST_NEXT                                    \
    "SX%=:\n\t" GP_FAST_XU GP_FAST_TU("sub") GP_FAST_NEXT                         \
    "SC%=:\n\t" GP_FAST_TC("sub") GP_FAST_NEXT                                    \
    "RX%=:\n\t" GP_FAST_XU GP_FAST_RSUB("%%u0", "%%u1", "%%u2", "%%u3") GP_FAST_NEXT \
    "RC%=:\n\t" GP_FAST_RSUB("%%cf", "%%cf", "%%cf", "%%cf") GP_FAST_NEXT         \
    "MX%=:\n\t" GP_FAST_XU GP_FAST_TU("mul") GP_FAST_NEXT                         \
    "MC%=:\n\t" GP_FAST_TC("mul") GP_FAST_NEXT                                    \
    "AB%=:\n\t"                                                                   \
    "abs.f32 %1, %1;\n\tabs.f32 %2, %2;\n\tabs.f32 %3, %3;\n\tabs.f32 %4, %4;\n\t" \
    GP_FAST_NEXT                                                                  \
    "NG%=:\n\t"                                                                   \
    "neg.f32 %1, %1;\n\tneg.f32 %2, %2;\n\tneg.f32 %3, %3;\n\tneg.f32 %4, %4;\n\t" \
    GP_FAST_NEXT                                                                  \
    "EX%=:\n\t"                                                                   \
    "mov.b32 %5, %%w;\n\t"                                                        \
    "mov.f32 %6, %%cf;\n\t"                                                       \
    "}\n"

// XREG: columns 0 and 1 held in x0 and x1 (otherwise those are unused and
// the column reads are handed back)
#define GP_FAST_OPERANDS                                                          \
    : "+r"(pa), "+f"(t[0]), "+f"(t[1]), "+f"(t[2]), "+f"(t[3]), "=r"(hw), "=f"(hc) \
    : "r"(sb), "n"(NSLOT - 1), "f"(x0[0]), "f"(x0[1]), "f"(x0[2]), "f"(x0[3]),    \
      "f"(x1[0]), "f"(x1[1]), "f"(x1[2]), "f"(x1[3]), "f"(kThr)                   \
    : "memory"
template <int NSLOT, bool DIVS, bool XREG>
__device__ __forceinline__ void run_fast4(uint32_t &pa, float (&t)[4], const float (&x0)[4],
                                          const float (&x1)[4], uint32_t sb, uint32_t &hw,
                                          float &hc) {
    if constexpr (!XREG && DIVS) {
        asm volatile(GP_FAST_HEAD(GP_FAST_TABLE_DIVS_NOX) GP_FAST_TRIG_REGS GP_FAST_DIV_BODIES
                     GP_FAST_TRIG_BODIES GP_FAST_BODY GP_FAST_OPERANDS);
    } else if constexpr (!XREG) {
        asm volatile(GP_FAST_HEAD(GP_FAST_TABLE_NODIVS_NOX) GP_FAST_BODY GP_FAST_OPERANDS);
    } else if constexpr (DIVS) {
        asm volatile(GP_FAST_HEAD(GP_FAST_TABLE_DIVS) GP_FAST_TRIG_REGS GP_FAST_DIV_BODIES
                     GP_FAST_TRIG_BODIES GP_FAST_BODY
                     : "+r"(pa), "+f"(t[0]), "+f"(t[1]), "+f"(t[2]), "+f"(t[3]), "=r"(hw),
                       "=f"(hc)
                     : "r"(sb), "n"(NSLOT - 1), "f"(x0[0]), "f"(x0[1]), "f"(x0[2]), "f"(x0[3]),
                       "f"(x1[0]), "f"(x1[1]), "f"(x1[2]), "f"(x1[3]), "f"(kThr)
                     : "memory");
    } else {
        asm volatile(GP_FAST_HEAD(GP_FAST_TABLE_NODIVS) GP_FAST_BODY
                     : "+r"(pa), "+f"(t[0]), "+f"(t[1]), "+f"(t[2]), "+f"(t[3]), "=r"(hw),
                       "=f"(hc)
                     : "r"(sb), "n"(NSLOT - 1), "f"(x0[0]), "f"(x0[1]), "f"(x0[2]), "f"(x0[3]),
                       "f"(x1[0]), "f"(x1[1]), "f"(x1[2]), "f"(x1[3])
                     : "memory");
    }
}
#undef GP_FAST_HEAD
#undef GP_FAST_TABLE_DIVS
#undef GP_FAST_TABLE_NODIVS
#undef GP_FAST_TABLE_DIVS_NOX
#undef GP_FAST_TABLE_NODIVS_NOX
#undef GP_FAST_OPERANDS
#undef GP_FAST_LOOP_TOP
#undef GP_FAST_DIV_BODIES
#undef GP_FAST_TRIG_REGS
#undef GP_FAST_TRIG_CHECK1
#undef GP_FAST_TRIG_CHECK
#undef GP_FAST_TRIG_POLY
#undef GP_FAST_SINCOS1
#undef GP_FAST_TAN1
#undef GP_FAST_TRIG_BODIES
#undef GP_FAST_SLOT
#undef GP_FAST_SPILL
#undef GP_FAST_SLOTLOAD
#undef GP_FAST_X
#undef GP_FAST_XU
#undef GP_FAST_TV
#undef GP_FAST_TU
#undef GP_FAST_TC
#undef GP_FAST_RSUB
#undef GP_FAST_DIV1
#undef GP_FAST_DIV_TV
#undef GP_FAST_DIV_VT
#undef GP_FAST_SQRT1
#undef GP_FAST_INV1
#undef GP_FAST_SETC
#undef GP_FAST_NEXT
#undef GP_FAST_BODY

// Runs one compiled program over RPT rows per lane; returns the top of the
// stack in t.  stk = this warp's stack slice, already offset by the lane.
// The instruction buffer (kCodeStride + 2 entries in shared memory, one
// more than either loop can reach) holds OP_END from the program's end
// through its last entry, so the loop ends within kCodeStride + 1 steps
// whatever the buffer holds; op values that name no operation act as
// OP_END and stack slots are clamped to the stack, so no instruction word
// can make it run away or leave its memory.
//
// Dispatch cost is what this loop is tuned for (per-opcode instruction
// counts measured with ncu on chains of one operation).  At 4 rows per lane
// the fast loop runs most words and hands the others, one at a time, to
// the switch below.  The instruction word and the stack are addressed
// through 32-bit shared-memory addresses computed once; the opcode is
// broadcast from lane 0, which lets the compiler treat the switch as
// warp-uniform (no reconvergence barrier per instruction); the switch
// covers all 32 values of its 5-bit operand, so it needs no range test;
// and the word is loaded when it is needed rather than one ahead, which
// saves the register copies of a prefetch.
template <int RPT, int NSLOT, int FMODE, bool EXT>
__device__ __forceinline__ void interpret(float (&t)[RPT], const uint2 *__restrict__ cbuf,
                                          const float (&x0)[RPT], const float (&x1)[RPT],
                                          const float *__restrict__ X, int64_t ld, int64_t r0,
                                          int64_t re, bool vec, float4 *stk) {
    // EXT: the extended functions are compiled in (classes 1 and 2).  In
    // class 0, where nearly all programs of the usual function set run,
    // their cases cost 2-3% (measured on Pagie-1 x 4096 programs, which
    // never use them)
    constexpr bool kExt = EXT;
#pragma unroll
    for (int j = 0; j < RPT; ++j) t[j] = 0.0f;
    // pa: shared-memory address of the next instruction word
    uint32_t pa = (uint32_t)__cvta_generic_to_shared(cbuf);
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(stk);  // this lane's slot 0
    // 4 rows per lane: the fast loop runs what it can and hands back the
    // rest, one word at a time, to the switch below
    constexpr bool kFast = RPT == 4;
#pragma unroll 1
    for (;;) {
        uint2 ins;
        if constexpr (kFast) {
            float hc;
            run_fast4<NSLOT, !EXT, FMODE == 2>(pa, t, x0, x1, sb, ins.x, hc);
            ins.y = __float_as_uint(hc);
        } else {
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                         : "=r"(ins.x), "=r"(ins.y)
                         : "r"(pa));
            pa += 8u;
        }
        const uint32_t w = __shfl_sync(0xffffffffu, ins.x, 0);
        const float c = __uint_as_float(ins.y);
// operand helpers: stack slot, X column, constant
// (the stack is laid out [slot][q][lane] in float4: slot sl, group q of
// this lane sits (sl * RPT/4 + q) * 32 float4 past its slot 0)
#define GP_SLOT_LOAD(u)                                                         \
    {                                                                           \
        const uint32_t sl = min((w >> 8) & 255u, (uint32_t)NSLOT - 1u);         \
        _Pragma("unroll") for (int q = 0; q < RPT / 4; ++q) {                   \
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"             \
                         : "=f"(u[4 * q]), "=f"(u[4 * q + 1]),                  \
                           "=f"(u[4 * q + 2]), "=f"(u[4 * q + 3])               \
                         : "r"(sb + (sl * (RPT / 4) + q) * 32u * 16u));          \
        }                                                                       \
    }
#define GP_SPILL()                                                              \
    {                                                                           \
        const uint32_t sl = min((w >> 8) & 255u, (uint32_t)NSLOT - 1u);         \
        _Pragma("unroll") for (int q = 0; q < RPT / 4; ++q)                     \
            asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"             \
                         ::"r"(sb + (sl * (RPT / 4) + q) * 32u * 16u),           \
                           "f"(t[4 * q]), "f"(t[4 * q + 1]), "f"(t[4 * q + 2]),  \
                           "f"(t[4 * q + 3])                                    \
                         : "memory");                                           \
    }
#define GP_X_LOAD(u)                                                            \
    {                                                                           \
        const int feat = (int)(w >> 16);                                        \
        if (FMODE == 2) {                                                       \
            _Pragma("unroll") for (int j = 0; j < RPT; ++j) u[j] = feat ? x1[j] : x0[j]; \
        } else {                                                                \
            load_rows<RPT>(u, X + (int64_t)feat * ld, r0, re, vec);             \
        }                                                                       \
    }
#define GP_T(expr) _Pragma("unroll") for (int j = 0; j < RPT; ++j) t[j] = expr;
#define GP_U_C(u) _Pragma("unroll") for (int j = 0; j < RPT; ++j) u[j] = c;
        float u[RPT];
        switch (w & 31u) {
            case OP_PUSH_X: GP_X_LOAD(u) GP_T(u[j]) break;
            case OP_PUSH_C: GP_T(c) break;
            case OP_PUSH_X_SP: GP_SPILL() GP_X_LOAD(u) GP_T(u[j]) break;
            case OP_PUSH_C_SP: GP_SPILL() GP_T(c) break;
            case OP_ADD_S: GP_SLOT_LOAD(u) GP_T(f_add(t[j], u[j])) break;
            case OP_SUB_S: GP_SLOT_LOAD(u) GP_T(f_sub(t[j], u[j])) break;
            case OP_MUL_S: GP_SLOT_LOAD(u) GP_T(f_mul(t[j], u[j])) break;
            case OP_DIV_S: GP_SLOT_LOAD(u) goto div_tu;
            case OP_ADD_X: GP_X_LOAD(u) GP_T(f_add(t[j], u[j])) break;
            case OP_ADD_C: GP_T(f_add(t[j], c)) break;
            case OP_SUB_X: GP_X_LOAD(u) GP_T(f_sub(t[j], u[j])) break;
            case OP_SUB_C: GP_T(f_sub(t[j], c)) break;
            case OP_RSUB_X: GP_X_LOAD(u) GP_T(f_sub(u[j], t[j])) break;
            case OP_RSUB_C: GP_T(f_sub(c, t[j])) break;
            case OP_MUL_X: GP_X_LOAD(u) GP_T(f_mul(t[j], u[j])) break;
            case OP_MUL_C: GP_T(f_mul(t[j], c)) break;
            case OP_DIV_X: GP_X_LOAD(u) goto div_tu;
            case OP_DIV_C: GP_U_C(u) goto div_tu;
            case OP_RDIV_X: GP_X_LOAD(u) goto div_ut;
            case OP_RDIV_C: GP_U_C(u) goto div_ut;
            case OP_SQRT: GP_T(f_sqrt(t[j])) break;
            case OP_LOG: GP_T(f_log(t[j])) break;
            case OP_EXP: GP_T(f_exp(t[j])) break;
            case OP_SIN:
            case OP_COS:
            case OP_TAN: trig_rows<RPT>(t, (int)(w & 31u) - OP_SIN); break;
            case OP_ABS: GP_T(f_abs(t[j])) break;
            case OP_NEG: GP_T(f_neg(t[j])) break;
            case OP_INV: GP_T(f_inv(t[j])) break;
            case OP_EXT1:  // out of line, four rows per call
                if constexpr (kExt) {
                    _Pragma("unroll") for (int g = 0; g < RPT / 4; ++g) {
                        const float4 r = ext_rows4(
                            make_float4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3]),
                            (w >> 5) & 7u);
                        t[4 * g] = r.x; t[4 * g + 1] = r.y; t[4 * g + 2] = r.z; t[4 * g + 3] = r.w;
                    }
                    break;
                } else {
                    goto done;
                }
            case OP_EXT2:  // max / min, right operand in a stack slot
                if constexpr (kExt) {
                    GP_SLOT_LOAD(u)
                    if (((w >> 5) & 7u) == EXT_MAX) { GP_T(f_max(t[j], u[j])) }
                    else { GP_T(f_min(t[j], u[j])) }
                    break;
                } else {
                    goto done;
                }
            case OP_END:
                goto done;
            default:  // every value of w & 31 has a case above
                __builtin_unreachable();
        }
        continue;
        // division has one body per operand order, shared by its operand cases
    div_tu:
        GP_T(f_div(t[j], u[j]))
        continue;
    div_ut:
        GP_T(f_div(u[j], t[j]))
#undef GP_T
#undef GP_U_C
#undef GP_X_LOAD
#undef GP_SPILL
#undef GP_SLOT_LOAD
    }
done:;
}

// shared memory of one block: the program's instructions, then the stack
template <int RPT, int NSLOT>
constexpr size_t eval_smem_bytes() {
    return (size_t)(kCodeStride + 2) * sizeof(uint2) +
           (size_t)eval_warps<RPT>() * NSLOT * (RPT / 4) * 32 * sizeof(float4);
}

// epilogues: the weighted loss sum, the predictions, or the moment sums
// of the correlation fitness.  The moment epilogue asks for the loss
// epilogue's occupancy: 5 resident blocks at 4 rows per thread (at most 48
// registers, with a few spilled words: 4% faster than 4 blocks at 59
// registers on Pagie-1 16M x 4096) and 3 at 8 rows (at most 85 registers;
// left alone it would take 97 and fit 2).
constexpr int kEpiLoss = 0, kEpiPred = 1, kEpiMom = 2;

template <int RPT, int NSLOT, int FMODE, int EPI, bool EXT>
__global__ void __launch_bounds__(eval_warps<RPT>() * 32, EPI == kEpiMom ? (RPT == 8 ? 3 : 5) : 0) eval_kernel(const EvalArgs a) {
    constexpr bool PRED = EPI == kEpiPred;
    constexpr bool MOM = EPI == kEpiMom;
    constexpr int kEvalWarps = eval_warps<RPT>();
    constexpr int kEvalBlock = kEvalWarps * 32;
    extern __shared__ float4 smem_eval[];
    uint2 *cbuf = reinterpret_cast<uint2 *>(smem_eval);
    float4 *stack_all = smem_eval + ((kCodeStride + 2) * sizeof(uint2) + 15) / 16;
    __shared__ float wsum[kEvalWarps];
    __shared__ double wmom[MOM ? kEvalWarps : 1][3];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4 *stk = stack_all + (size_t)warp * NSLOT * (RPT / 4) * 32 + lane;
    const int cls_begin = (a.cls == 0) ? 0 : a.class_count[0] + (a.cls == 2 ? a.class_count[1] : 0);
    const int n_cls = a.class_count[a.cls];
    const unsigned long long total = (unsigned long long)n_cls * (unsigned long long)a.n_chunks;
    const bool vec = a.vec_ok != 0;
    const bool two_feat = FMODE == 2 && a.ld > 0;
    const float ybar = MOM ? (float)a.ystat[3] : 0.0f;

    for (unsigned long long it = 0; it <= total; ++it) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1ULL);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= total || it == total) {  // the cap cannot trigger: one item per pass
            if (it == total && threadIdx.x == 0) atomicOr(a.dev_status, GP_DEV_QUEUE_CAP);
            break;
        }
        const int chunk = (int)(item / (unsigned long long)n_cls);
        const int rank = (int)(item - (unsigned long long)chunk * n_cls);
        const int p = a.order[cls_begin + rank];
        const ProgMeta m = a.meta[p];
        const int64_t rb = (int64_t)chunk * a.chunk_rows;
        const int64_t re = min(a.n_rows, rb + a.chunk_rows);

        if (m.status != GP_PROG_OK) {
            if (PRED) {
                for (int64_t r = rb + threadIdx.x; r < re; r += kEvalBlock)
                    a.pred[(size_t)p * a.n_rows + r] = __int_as_float(0x7fc00000);
            } else if (MOM) {
                if (threadIdx.x < 3)
                    a.mom[((size_t)p * a.n_chunks + chunk) * 3 + threadIdx.x] =
                        __longlong_as_double(0x7ff8000000000000LL);
            } else if (threadIdx.x == 0) {
                a.part[(size_t)p * a.n_chunks + chunk] = __int_as_float(0x7fc00000);
            }
            __syncthreads();  // s_item is rewritten at the top
            continue;
        }
        // the program, then OP_END through the buffer's last entry (the last
        // one stored apart: as a third pass of the loop it cost the kernel
        // 15 registers)
        for (int i = threadIdx.x; i <= kCodeStride; i += kEvalBlock)
            cbuf[i] = (i < m.n_ins) ? a.code[(size_t)p * kCodeStride + i]
                                    : make_uint2(make_ins(OP_END, 0, 0), 0u);
        if (threadIdx.x == 0) cbuf[kCodeStride + 1] = make_uint2(make_ins(OP_END, 0, 0), 0u);
        __syncthreads();

        float ks = 0.0f, kc = 0.0f;
        float ms[3] = {0.0f, 0.0f, 0.0f}, mc[3] = {0.0f, 0.0f, 0.0f};
        const float shift = MOM ? a.shift[p] : 0.0f;
        for (int64_t base = rb + (int64_t)warp * 32 * RPT; base < re;
             base += (int64_t)kEvalWarps * 32 * RPT) {
            const int64_t r0 = base + (int64_t)lane * RPT;
            float x0[RPT], x1[RPT];
            if (FMODE == 2) {
                load_rows<RPT>(x0, a.X, r0, re, vec);
                if (two_feat) load_rows<RPT>(x1, a.X + a.ld, r0, re, vec);
                else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) x1[j] = x0[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < RPT; ++j) x0[j] = x1[j] = 0.0f;
            }
            float t[RPT];
            interpret<RPT, NSLOT, FMODE, EXT>(t, cbuf, x0, x1, a.X, a.ld, r0, re, vec, stk);
            if (PRED) {
                float *dst = a.pred + (size_t)p * a.n_rows;
#pragma unroll
                for (int j = 0; j < RPT; ++j)
                    if (r0 + j < re) dst[r0 + j] = t[j];
            } else if (MOM) {
                // d = p - shift keeps the sums of squares free of the
                // cancellation a large mean would cause
                float yv[RPT], wv[RPT];
                load_rows<RPT>(yv, a.y, r0, re, vec);
                if (a.w) load_rows<RPT>(wv, a.w, r0, re, vec);
                float e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const float d = __fsub_rn(t[j], shift);
                    const float yc = __fsub_rn(yv[j], ybar);
                    const float wd = a.w ? __fmul_rn(wv[j], d) : d;
                    const bool in = r0 + j < re;
                    e1 = in ? __fadd_rn(e1, wd) : e1;
                    e2 = in ? __fadd_rn(e2, __fmul_rn(wd, d)) : e2;
                    e3 = in ? __fadd_rn(e3, __fmul_rn(wd, yc)) : e3;
                }
                kahan_add(ms[0], mc[0], e1);
                kahan_add(ms[1], mc[1], e2);
                kahan_add(ms[2], mc[2], e3);
            } else {
                float yv[RPT], wv[RPT];
                load_rows<RPT>(yv, a.y, r0, re, vec);
                if (a.w) load_rows<RPT>(wv, a.w, r0, re, vec);
                float e = 0.0f;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    float l = row_loss(a.metric, t[j], yv[j]);
                    if (a.w) l = __fmul_rn(wv[j], l);
                    e = (r0 + j < re) ? __fadd_rn(e, l) : e;
                }
                kahan_add(ks, kc, e);
            }
        }
        if (MOM) {
            // the lane's compensated sums in FP64, then a fixed butterfly
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double v = (double)ms[k] - (double)mc[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) wmom[warp][k] = v;
            }
        } else if (!PRED) {
            float v = __fsub_rn(ks, kc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) wsum[warp] = v;
        }
        __syncthreads();  // wsum complete; everyone is done with cbuf and s_item
        if (MOM && threadIdx.x < 3) {
            double v = 0.0;
            for (int w = 0; w < kEvalWarps; ++w) v += wmom[w][threadIdx.x];
            a.mom[((size_t)p * a.n_chunks + chunk) * 3 + threadIdx.x] = v;
        } else if (!PRED && !MOM && threadIdx.x == 0) {
            float v = 0.0f;
            for (int w = 0; w < kEvalWarps; ++w) v = __fadd_rn(v, wsum[w]);
            a.part[(size_t)p * a.n_chunks + chunk] = v;
        }
    }
}

template <int RPT, int NSLOT, int FMODE, int EPI, bool EXT>
cudaError_t launch_eval_t(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    (void)block;
    constexpr size_t smem = eval_smem_bytes<RPT, NSLOT>();
    auto k = eval_kernel<RPT, NSLOT, FMODE, EPI, EXT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, eval_warps<RPT>() * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RPT, int NSLOT, int FMODE, int EPI, bool EXT>
int info_t(int block, int *regs) {
    (void)block;
    constexpr size_t smem = eval_smem_bytes<RPT, NSLOT>();
    auto k = eval_kernel<RPT, NSLOT, FMODE, EPI, EXT>;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
    if (regs) *regs = fa.numRegs;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, eval_warps<RPT>() * 32, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace gpk
