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
#include "gp_fast.cuh"

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
    // the logarithm sees max(|a|, thr); inf and NaN, for which both tests
    // fail, are passed through
    const float b = fabsf(a);
    const float l = log_pos(fmaxf(b, kThr));
    return b < kThr ? 0.0f : (b <= 3.40282347e38f ? l : b);
}
__device__ __forceinline__ float f_exp(float a) {
    if (fabsf(a) < kExpFast) return exp_fast(a);
    if (a >= kExpInf) return __int_as_float(0x7f800000);
    return a <= kExpZero ? 0.0f : exp_wide(a);  // NaN: NaN
}
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

// RPT consecutive rows of one column from p; with vec all of them as
// 16-byte loads, otherwise the first nv rows one by one and 0 after them
template <int RPT>
__device__ __forceinline__ void load_chunk_rows(float (&v)[RPT], const float *__restrict__ p,
                                                bool vec, int nv) {
    if (vec) {
#pragma unroll
        for (int q = 0; q < RPT / 4; ++q) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(p) + q);
            v[4 * q + 0] = f.x;
            v[4 * q + 1] = f.y;
            v[4 * q + 2] = f.z;
            v[4 * q + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < RPT; ++j) v[j] = (j < nv) ? __ldg(p + j) : 0.0f;
    }
}

// the weighted losses of a lane's rows added in row order (the first nv
// rows count); the metric and the weights are tested once, not per row
template <int RPT>
__device__ __forceinline__ float loss_sum(int metric, const float (&t)[RPT],
                                          const float (&yv)[RPT], const float (&wv)[RPT],
                                          bool has_w, bool full, int nv) {
    float l[RPT];
    if (metric == GP_MAE) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) l[j] = row_loss(GP_MAE, t[j], yv[j]);
    } else if (metric == GP_LOGLOSS) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) l[j] = row_loss(GP_LOGLOSS, t[j], yv[j]);
    } else {
#pragma unroll
        for (int j = 0; j < RPT; ++j) l[j] = row_loss(GP_MSE, t[j], yv[j]);
    }
    if (has_w) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) l[j] = __fmul_rn(wv[j], l[j]);
    }
    float e = 0.0f;
    if (full) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) e = __fadd_rn(e, l[j]);
    } else {
#pragma unroll
        for (int j = 0; j < RPT; ++j) e = (j < nv) ? __fadd_rn(e, l[j]) : e;
    }
    return e;
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
// 3).  gp_fast.cuh (written by gen_fast.py) holds the loop for 4 and 8 rows
// per lane: a lane's rows sit in RPT/2 64-bit pairs and add, sub, mul and
// fma run as one packed f32x2 instruction per pair (per-element round to
// nearest, no flush to zero: the bits of the scalar operations).  It runs
// pushes and stack moves, add/sub/mul with every operand form, abs, neg,
// column reads from registers (XREG) and, with DIVS, the protected
// divisions, square root, reciprocal, sin, cos, tan, log and exp (the steps
// and constants of gp_math.cuh, so results are the same bits).  It stops
// at the first word it does not run (END, the extended functions, a
// trigonometric or exponential argument outside the fast path in any row
// of the warp, and whatever XREG or DIVS leave out), hands that word and
// its constant back to the switch below and leaves pa just past it.  DIVS
// is off in the instances with the extended functions: there the division
// set in the loop cost the extended-set population 23% (their out-of-line
// calls and the division's own slow-path call do not mix well).
__device__ __forceinline__ uint64_t pack2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}

template <int RPT, int NSLOT, bool DIVS, bool XREG>
__device__ __forceinline__ void run_fast(uint32_t &pa, uint64_t (&t)[RPT / 2],
                                         const uint64_t (&x0)[RPT / 2],
                                         const uint64_t (&x1)[RPT / 2], uint32_t sb,
                                         uint32_t &hw, float &hc) {
    if constexpr (RPT == 4) {
        if constexpr (DIVS && XREG) fast_r4_divs_x<NSLOT>(pa, t, x0, x1, sb, hw, hc);
        else if constexpr (DIVS) fast_r4_divs_nox<NSLOT>(pa, t, x0, x1, sb, hw, hc);
        else if constexpr (XREG) fast_r4_nodivs_x<NSLOT>(pa, t, x0, x1, sb, hw, hc);
        else fast_r4_nodivs_nox<NSLOT>(pa, t, x0, x1, sb, hw, hc);
    } else {
        if constexpr (DIVS && XREG) fast_r8_divs_x<NSLOT>(pa, t, x0, x1, sb, hw, hc);
        else if constexpr (DIVS) fast_r8_divs_nox<NSLOT>(pa, t, x0, x1, sb, hw, hc);
        else if constexpr (XREG) fast_r8_nodivs_x<NSLOT>(pa, t, x0, x1, sb, hw, hc);
        else fast_r8_nodivs_nox<NSLOT>(pa, t, x0, x1, sb, hw, hc);
    }
}

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
// counts measured with ncu on chains of one operation).  At 4 and 8 rows
// per lane the fast loop runs most words and hands the others, one at a
// time, to the switch below.  The instruction word and the stack are addressed
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
    // 4 or 8 rows per lane: the fast loop runs what it can and hands back
    // the rest, one word at a time, to the switch below; the rows cross
    // between the two as pairs {row 2i, row 2i+1} (register moves)
    constexpr bool kFast = RPT == 4 || RPT == 8;
    constexpr int kPairs = kFast ? RPT / 2 : 1;
    uint64_t x0p[kPairs], x1p[kPairs];
    if constexpr (kFast) {
#pragma unroll
        for (int i = 0; i < kPairs; ++i) {
            x0p[i] = pack2(x0[2 * i], x0[2 * i + 1]);
            x1p[i] = pack2(x1[2 * i], x1[2 * i + 1]);
        }
    }
#pragma unroll 1
    for (;;) {
        uint2 ins;
        if constexpr (kFast) {
            float hc;
            uint64_t tp[kPairs];
#pragma unroll
            for (int i = 0; i < kPairs; ++i) tp[i] = pack2(t[2 * i], t[2 * i + 1]);
            run_fast<RPT, NSLOT, !EXT, FMODE == 2>(pa, tp, x0p, x1p, sb, ins.x, hc);
#pragma unroll
            for (int i = 0; i < kPairs; ++i) unpack2(tp[i], t[2 * i], t[2 * i + 1]);
            ins.y = __float_as_uint(hc);
        } else {
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                         : "=r"(ins.x), "=r"(ins.y)
                         : "r"(pa));
            pa += 8u;
        }
        const uint32_t w = __shfl_sync(0xffffffffu, ins.x, 0);
        // the end of the program, once per sub-tile: out before the switch
        if ((w & 31u) == OP_END) break;
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
                            (w >> 16) & 7u);
                        t[4 * g] = r.x; t[4 * g + 1] = r.y; t[4 * g + 2] = r.z; t[4 * g + 3] = r.w;
                    }
                    break;
                } else {
                    goto done;
                }
            case OP_EXT2:  // max / min, right operand in a stack slot
                if constexpr (kExt) {
                    GP_SLOT_LOAD(u)
                    if (((w >> 16) & 7u) == EXT_MAX) { GP_T(f_max(t[j], u[j])) }
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
// of the correlation fitness.  At 8 rows per thread the loss and store
// epilogues ask for 4 resident blocks (at most 64 registers, with the
// 6-slot stack of class 0: 295 against 312 ms at 3 blocks on Pagie-1 16M
// x 4096), the moment epilogue for 3 (at most 85 registers).  At 4 rows the moment epilogue asks for 5 (at most 48
// registers, a few spilled words: 4% faster than 4 blocks at 59 registers
// on Pagie-1 16M x 4096); the others are left alone (46 registers: 5 fit),
// because asking for 5 blocks there changed their schedule and cost 7%.
constexpr int kEpiLoss = 0, kEpiPred = 1, kEpiMom = 2;

template <int RPT, int NSLOT, int FMODE, int EPI, bool EXT>
__global__ void __launch_bounds__(eval_warps<RPT>() * 32,
                                  RPT == 8 ? (EPI == kEpiMom ? 3 : 4)
                                           : (EPI == kEpiMom && RPT == 4 ? 5 : 0))
    eval_kernel(const EvalArgs a) {
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
    const int qc = a.qcls ? a.qcls - 1 : a.cls;  // the span of the program order
    int cls_begin = 0;
    for (int b = 0; b < qc; ++b) cls_begin += a.class_count[b];
    int n_cls = a.class_count[qc];
    if (a.sub == 1) {  // the long programs of class 0 (first in its order)
        n_cls = a.class_count[kOrderClasses];
    } else if (a.sub == 2) {  // the rest of class 0
        cls_begin = a.class_count[kOrderClasses];
        n_cls -= cls_begin;
    }
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
        const uint2 *src = a.code + (size_t)p * (a.code_stride ? a.code_stride : kCodeStride);
        for (int i = threadIdx.x; i <= kCodeStride; i += kEvalBlock)
            cbuf[i] = (i < m.n_ins) ? src[i] : make_uint2(make_ins(OP_END, 0, 0), 0u);
        if (threadIdx.x == 0) cbuf[kCodeStride + 1] = make_uint2(make_ins(OP_END, 0, 0), 0u);
        __syncthreads();

        float ks = 0.0f, kc = 0.0f;
        float ms[3] = {0.0f, 0.0f, 0.0f}, mc[3] = {0.0f, 0.0f, 0.0f};
        const float shift = MOM ? a.shift[p] : 0.0f;
        // rows of the chunk in 32-bit offsets from its first row (a chunk
        // holds at most 2^30 rows); pointers to the chunk's columns once
        const int n_in = (int)(re - rb);
        // the column pointers are formed per use from the kernel arguments
        // (held in constant memory): four live 64-bit pointers would cost
        // the loop 8 registers and a resident block
        const int64_t x1off = two_feat ? a.ld : 0;
        for (int base = warp * 32 * RPT; base < n_in; base += kEvalWarps * 32 * RPT) {
            const int o = base + lane * RPT;  // this lane's first row in the chunk
            // every row of the warp is in the chunk except in its last
            // sub-tile; decided once for the warp (a vote), so the loads and
            // the loss take no divergent branch (each per-lane test had cost
            // a reconvergence barrier pair per sub-tile)
            const bool full = __all_sync(0xffffffffu, o + RPT <= n_in);
            const int nv = full ? RPT : n_in - o;  // rows of the lane to count
            float x0[RPT], x1[RPT];
            if (FMODE == 2) {
                load_chunk_rows<RPT>(x0, a.X + (rb + o), full && vec, nv);
                if (two_feat) load_chunk_rows<RPT>(x1, a.X + (x1off + rb + o), full && vec, nv);
                else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) x1[j] = x0[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < RPT; ++j) x0[j] = x1[j] = 0.0f;
            }
            float t[RPT];
            interpret<RPT, NSLOT, FMODE, EXT>(t, cbuf, x0, x1, a.X, a.ld, rb + o, re, vec, stk);
            if (PRED) {
                float *dst = a.pred + (size_t)p * a.n_rows + rb + o;
#pragma unroll
                for (int j = 0; j < RPT; ++j)
                    if (j < nv) dst[j] = t[j];
            } else if (MOM) {
                // d = p - shift keeps the sums of squares free of the
                // cancellation a large mean would cause
                float yv[RPT], wv[RPT];
                load_chunk_rows<RPT>(yv, a.y + (rb + o), full && vec, nv);
                if (a.w) load_chunk_rows<RPT>(wv, a.w + (rb + o), full && vec, nv);
                float e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const float d = __fsub_rn(t[j], shift);
                    const float yc_ = __fsub_rn(yv[j], ybar);
                    const float wd = a.w ? __fmul_rn(wv[j], d) : d;
                    const bool in = j < nv;
                    e1 = in ? __fadd_rn(e1, wd) : e1;
                    e2 = in ? __fadd_rn(e2, __fmul_rn(wd, d)) : e2;
                    e3 = in ? __fadd_rn(e3, __fmul_rn(wd, yc_)) : e3;
                }
                kahan_add(ms[0], mc[0], e1);
                kahan_add(ms[1], mc[1], e2);
                kahan_add(ms[2], mc[2], e3);
            } else {
                float yv[RPT], wv[RPT];
                load_chunk_rows<RPT>(yv, a.y + (rb + o), full && vec, nv);
                if (a.w) load_chunk_rows<RPT>(wv, a.w + (rb + o), full && vec, nv);
                kahan_add(ks, kc, loss_sum<RPT>(a.metric, t, yv, wv, a.w != nullptr, full, nv));
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
