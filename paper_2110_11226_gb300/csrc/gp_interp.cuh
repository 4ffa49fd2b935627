// gp_interp.cuh -- the batched persistent evaluator (the hot loop).
//
// Work: every (program, row-chunk) pair of one depth class is an item of a
// dynamic queue (one atomic counter); items are ordered chunk-major and,
// inside a chunk, longest program first, so the warps that share the GPU
// at any moment work on the same few row chunks (X stays in L2) and the
// queue drains with the short items last.
//
// A warp takes one item: it copies the program's compiled instructions
// into its slice of shared memory, then walks the chunk in sub-tiles of
// 32*RPT rows.  Lane l owns rows base + l*RPT .. +RPT-1 (vectorised,
// coalesced loads from the column-major X).  The instruction stream is the
// same for all 32 lanes, so the switch below is warp-uniform: the
// execution kernel of Sec. III-C3 needs every thread of a block on one
// program to avoid divergence; here one warp is enough.  The stack is the
// register arrays t[RPT] (top) and s[MAXD][RPT] (deeper slots), addressed
// only with compile-time indices.
//
// After a sub-tile each lane turns its RPT predictions into weighted losses
// (the fused form of the paper's matrix-vector loss step), adds them into a
// Kahan-compensated FP32 sum, and at the end of the item the warp adds the
// 32 lane sums with a fixed butterfly; lane 0 writes one partial per
// (program, chunk).  A separate pass adds the partials of a program in
// chunk order in FP64.  Every step has a fixed order, so results do not
// depend on which warp ran which item.
#pragma once

#include "gp_internal.cuh"
#include "gp_math.cuh"

namespace gpk {

constexpr int kEvalBlock = kEvalBlockThreads;

// ---- the function set (FP32, IEEE operators, no contraction) -----------
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_div(float a, float b) {
    return fabsf(b) < kThr ? 1.0f : __fdiv_rn(a, b);
}
__device__ __forceinline__ float f_sqrt(float a) { return __fsqrt_rn(fabsf(a)); }
__device__ __forceinline__ float f_log(float a) {
    const float b = fabsf(a);
    return b < kThr ? 0.0f : logf(b);
}
__device__ __forceinline__ float f_exp(float a) { return expf(a); }
__device__ __forceinline__ float f_sin(float a) { return sinf(a); }
__device__ __forceinline__ float f_cos(float a) { return cosf(a); }
__device__ __forceinline__ float f_tan(float a) { return tanf(a); }
__device__ __forceinline__ float f_abs(float a) { return fabsf(a); }
__device__ __forceinline__ float f_neg(float a) { return -a; }
__device__ __forceinline__ float f_inv(float a) {
    return fabsf(a) < kThr ? 0.0f : __frcp_rn(a);
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

template <int RPT>
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float yv = __fsub_rn(x, c);
    const float tv = __fadd_rn(s, yv);
    // once the sum is infinite or NaN the compensation is meaningless
    c = isfinite(tv) ? __fsub_rn(__fsub_rn(tv, s), yv) : 0.0f;
    s = tv;
}

#define GP_R19(M) M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) \
    M(11) M(12) M(13) M(14) M(15) M(16) M(17) M(18)
#define GP_R20(M) GP_R19(M) M(19)

template <int RPT, int MAXD, int FMODE, bool PRED>
__global__ void __launch_bounds__(kEvalBlock) eval_kernel(const EvalArgs a) {
    extern __shared__ uint2 smem_code[];
    const int lane = threadIdx.x & 31;
    uint2 *cbuf = smem_code + (threadIdx.x >> 5) * (kCodeStride + 1);
    const int cls_begin = (a.cls == 0) ? 0 : a.class_count[0];
    const int n_cls = a.class_count[a.cls];
    const unsigned long long total = (unsigned long long)n_cls * (unsigned long long)a.n_chunks;
    const bool vec = a.vec_ok != 0;
    const bool two_feat = FMODE == 2 && a.ld > 0;

    for (unsigned long long it = 0; it <= total; ++it) {
        if (it == total) {  // cannot happen: each iteration takes one item
            if (lane == 0) atomicOr(a.dev_status, GP_DEV_QUEUE_CAP);
            break;
        }
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int chunk = (int)(item / (unsigned long long)n_cls);
        const int rank = (int)(item - (unsigned long long)chunk * n_cls);
        const int p = a.order[cls_begin + rank];
        const ProgMeta m = a.meta[p];
        const int64_t rb = (int64_t)chunk * a.chunk_rows;
        const int64_t re = min(a.n_rows, rb + a.chunk_rows);

        if (m.status != GP_PROG_OK) {
            if (PRED) {
                for (int64_t r = rb + lane; r < re; r += 32)
                    a.pred[(size_t)p * a.n_rows + r] = __int_as_float(0x7fc00000);
            } else if (lane == 0) {
                a.part[(size_t)p * a.n_chunks + chunk] = __int_as_float(0x7fc00000);
            }
            continue;
        }
        __syncwarp();
        for (int i = lane; i < m.n_ins; i += 32) cbuf[i] = a.code[(size_t)p * kCodeStride + i];
        __syncwarp();

        float ks = 0.0f, kc = 0.0f;
        for (int64_t base = rb; base < re; base += 32 * RPT) {
            const int64_t r0 = base + (int64_t)lane * RPT;
            float x0[RPT], x1[RPT];
            if (FMODE == 2) {
                load_rows<RPT>(x0, a.X, r0, re, vec);
                if (two_feat) load_rows<RPT>(x1, a.X + a.ld, r0, re, vec);
                else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) x1[j] = x0[j];
                }
            }
            float t[RPT];
            float s[MAXD][RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) t[j] = 0.0f;

            // One indirect dispatch per instruction.  Operand-fetch cases are
            // a few register moves and jump to the operation bodies below,
            // each of which exists once, so the hot code stays small.
            uint2 ins = cbuf[0];
            for (int pc = 0; pc < m.n_ins; ++pc) {
                const uint2 nx = cbuf[pc + 1];
                const uint32_t op = ins.x & 0xffu;
                const float c = __uint_as_float(ins.y);
                float u[RPT];
                if (ins.x & kNeedsX) {
                    const int feat = (int)(ins.x >> 16);
                    if (FMODE == 2) {
#pragma unroll
                        for (int j = 0; j < RPT; ++j) u[j] = feat ? x1[j] : x0[j];
                    } else {
                        load_rows<RPT>(u, a.X + (int64_t)feat * a.ld, r0, re, vec);
                    }
                }
                switch (op) {
#define GP_SPILL(k)                                                             \
    if constexpr (k > 0 && k <= MAXD) {                                         \
        _Pragma("unroll") for (int j = 0; j < RPT; ++j) s[k > 0 ? k - 1 : 0][j] = t[j]; \
    }
#define GP_PUSH(k)                                                              \
    case K_PUSH_X + k: GP_SPILL(k) goto L_TU;                                   \
    case K_PUSH_C + k: GP_SPILL(k) goto L_TC;
                    GP_R20(GP_PUSH)
#undef GP_PUSH
#undef GP_SPILL
#define GP_FETCH(k)                                                             \
    if constexpr (k < MAXD) {                                                   \
        _Pragma("unroll") for (int j = 0; j < RPT; ++j) u[j] = s[k < MAXD ? k : 0][j]; \
    }
#define GP_BIN_0(k) case K_BIN + 0 * kDeepSlots + k: GP_FETCH(k) goto L_ADD;
#define GP_BIN_1(k) case K_BIN + 1 * kDeepSlots + k: GP_FETCH(k) goto L_SUB;
#define GP_BIN_2(k) case K_BIN + 2 * kDeepSlots + k: GP_FETCH(k) goto L_MUL;
#define GP_BIN_3(k) case K_BIN + 3 * kDeepSlots + k: GP_FETCH(k) goto L_DIV;
                    GP_R19(GP_BIN_0)
                    GP_R19(GP_BIN_1)
                    GP_R19(GP_BIN_2)
                    GP_R19(GP_BIN_3)
#undef GP_BIN_0
#undef GP_BIN_1
#undef GP_BIN_2
#undef GP_BIN_3
#undef GP_FETCH
                    case K_BIN_RX + 0: case K_BIN_LX + 0: goto L_ADD;
                    case K_BIN_RX + 1: goto L_SUB;
                    case K_BIN_LX + 1: goto L_RSUB;
                    case K_BIN_RX + 2: case K_BIN_LX + 2: goto L_MUL;
                    case K_BIN_RX + 3: goto L_DIV;
                    case K_BIN_LX + 3: goto L_RDIV;
                    case K_BIN_RC + 0: case K_BIN_LC + 0: goto L_ADDC;
                    case K_BIN_RC + 1: goto L_SUBC;
                    case K_BIN_LC + 1: goto L_RSUBC;
                    case K_BIN_RC + 2: case K_BIN_LC + 2: goto L_MULC;
                    case K_BIN_RC + 3: goto L_DIVC;
                    case K_BIN_LC + 3: goto L_RDIVC;
#define GP_UN(i, fn)                                                            \
    case K_UN + i:                                                              \
        _Pragma("unroll") for (int j = 0; j < RPT; ++j) t[j] = fn(t[j]);        \
        goto L_NEXT;
                    GP_UN(0, f_sqrt)
                    GP_UN(1, f_log)
                    GP_UN(2, f_exp)
                    GP_UN(3, gp_sin)
                    GP_UN(4, gp_cos)
                    GP_UN(5, gp_tan)
                    GP_UN(6, f_abs)
                    GP_UN(7, f_neg)
                    GP_UN(8, f_inv)
#undef GP_UN
                    default:
                        goto L_END;  // K_END
                }
#define GP_BODY(label, expr)                                                    \
    label:                                                                      \
        _Pragma("unroll") for (int j = 0; j < RPT; ++j) t[j] = expr;            \
        goto L_NEXT;
                GP_BODY(L_TU, u[j])
                GP_BODY(L_TC, c)
                GP_BODY(L_ADD, f_add(t[j], u[j]))
                GP_BODY(L_SUB, f_sub(t[j], u[j]))
                GP_BODY(L_RSUB, f_sub(u[j], t[j]))
                GP_BODY(L_MUL, f_mul(t[j], u[j]))
                GP_BODY(L_DIV, f_div(t[j], u[j]))
                GP_BODY(L_RDIV, f_div(u[j], t[j]))
                GP_BODY(L_ADDC, f_add(t[j], c))
                GP_BODY(L_SUBC, f_sub(t[j], c))
                GP_BODY(L_RSUBC, f_sub(c, t[j]))
                GP_BODY(L_MULC, f_mul(t[j], c))
                GP_BODY(L_DIVC, f_div(t[j], c))
                GP_BODY(L_RDIVC, f_div(c, t[j]))
#undef GP_BODY
            L_NEXT:
                ins = nx;
            }
        L_END:
            if (PRED) {
                float *dst = a.pred + (size_t)p * a.n_rows;
#pragma unroll
                for (int j = 0; j < RPT; ++j)
                    if (r0 + j < re) dst[r0 + j] = t[j];
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
                kahan_add<RPT>(ks, kc, e);
            }
        }
        if (!PRED) {
            float v = __fsub_rn(ks, kc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) a.part[(size_t)p * a.n_chunks + chunk] = v;
        }
    }
}

template <int RPT, int MAXD, int FMODE, bool PRED>
cudaError_t launch_eval_t(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    const size_t smem = (size_t)(block / 32) * (kCodeStride + 1) * sizeof(uint2);
    auto k = eval_kernel<RPT, MAXD, FMODE, PRED>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RPT, int MAXD, int FMODE, bool PRED>
int info_t(int block, int *regs) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, eval_kernel<RPT, MAXD, FMODE, PRED>) != cudaSuccess) return 0;
    if (regs) *regs = fa.numRegs;
    const size_t smem = (size_t)(block / 32) * (kCodeStride + 1) * sizeof(uint2);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, eval_kernel<RPT, MAXD, FMODE, PRED>,
                                                      block, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace gpk
