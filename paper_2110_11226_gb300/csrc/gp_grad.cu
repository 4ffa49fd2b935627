// gp_grad.cu -- gradients of fitness with respect to the ephemeral
// constants (reverse mode), and one Adam step on the constants.  Neither
// has a counterpart in the paper; they serve constant tuning between
// generations.
//
// The adjoint runs on the compiled stack form of the evaluator
// (gp_internal.cuh), in its gradient variant: no constant-only subtree is
// folded, every word that reads a constant names the constant's slot, and
// every word that pops a stack slot names the word whose result was spilled
// into it.  A block takes one (program, row chunk) item; its warps run the
// program over their own sub-tiles of 32 * RPT rows:
//   forward   the words in order, as the evaluator runs them (the same FP32
//             operations, so the fitness equals gp_evaluate's), each word's
//             result written to the warp's tape in shared memory -- one float
//             per word and row, nothing of size programs x rows x nodes;
//   adjoint   the words in reverse: the adjoint of the top of the stack in
//             registers, the adjoints of spilled values in the warp's stack
//             slots (the forward values there are dead by then); a word's
//             input is the previous word's result on the tape, a popped
//             slot's value the spilled word's result; a word that reads a
//             constant adds its share to that constant's per-lane sum.
// Programs are bucketed by compiled length (kGradCap0, 1, 2, 256 words) and
// depth, one launch per bucket with a tape sized for its longest program.
// Per-lane sums are FP32 (the loss Kahan-compensated), warp sums
// fixed-order, chunk sums FP64 in order (gp_reduce.cu).
#include "gp_internal.cuh"
#include "gp_interp.cuh"

namespace gpk {

namespace {

__device__ __forceinline__ float sgnf(float x) {
    return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f);
}

// d loss / d p of one row (the metric readings of Sec. III-C3)
__device__ __forceinline__ float g_dloss(int metric, float p, float y) {
    if (metric == GP_MAE) return sgnf(__fsub_rn(p, y));
    if (metric == GP_LOGLOSS) {
        float s;
        if (p >= 0.0f) {
            s = __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-p)));
        } else {
            const float e = expf(p);
            s = __fdiv_rn(e, __fadd_rn(1.0f, e));
        }
        return __fsub_rn(s, y);
    }
    return __fmul_rn(2.0f, __fsub_rn(p, y));
}

// derivative of a unary word at input u with output v (the protected
// operators have derivative 0 on their protected branch)
__device__ __forceinline__ float d_unary(uint32_t op, uint32_t ext, float u, float v) {
    switch (op) {
    case OP_SQRT: return (u == 0.0f) ? 0.0f : __fdiv_rn(sgnf(u), __fmul_rn(2.0f, v));
    case OP_LOG: return fabsf(u) < kThr ? 0.0f : __frcp_rn(u);
    case OP_EXP: return v;
    case OP_SIN: return cosf(u);
    case OP_COS: return -sinf(u);
    case OP_TAN: return __fadd_rn(1.0f, __fmul_rn(v, v));
    case OP_ABS: return sgnf(u);
    case OP_NEG: return -1.0f;
    case OP_INV: return fabsf(u) < kThr ? 0.0f : -__fmul_rn(v, v);
    default:  // OP_EXT1
        switch (ext) {
        case EXT_SQ: return __fmul_rn(2.0f, u);
        case EXT_CUBE: return __fmul_rn(3.0f, __fmul_rn(u, u));
        case EXT_CBRT: return (u == 0.0f) ? 0.0f : __frcp_rn(__fmul_rn(3.0f, __fmul_rn(v, v)));
        case EXT_TANH: return __fsub_rn(1.0f, __fmul_rn(v, v));
        case EXT_ATAN: return __frcp_rn(__fadd_rn(1.0f, __fmul_rn(u, u)));
        case EXT_SINH: return coshf(u);
        default: return sinhf(u);  // EXT_COSH
        }
    }
}

// v into constant k's per-lane sum (k uniform over the warp).  Plain FP32:
// a lane adds at most 512 terms per 16K-row chunk (then FP64 across
// chunks); compensated sums had cost 16 registers and a resident block.
__device__ __forceinline__ void gadd(float (&gs)[GP_MAX_CONSTS], uint32_t k, float v) {
#define GP_GADD_CASE(q) \
    case q: gs[q] = __fadd_rn(gs[q], v); break;
    switch (k) {
        GP_GADD_CASE(0) GP_GADD_CASE(1) GP_GADD_CASE(2) GP_GADD_CASE(3)
        GP_GADD_CASE(4) GP_GADD_CASE(5) GP_GADD_CASE(6) GP_GADD_CASE(7)
        GP_GADD_CASE(8) GP_GADD_CASE(9) GP_GADD_CASE(10) GP_GADD_CASE(11)
        GP_GADD_CASE(12) GP_GADD_CASE(13) GP_GADD_CASE(14) GP_GADD_CASE(15)
        default: break;
    }
#undef GP_GADD_CASE
}

// the extended unary functions of one row (the evaluator's, so the forward
// values are its values)
__device__ __forceinline__ float f_ext1(uint32_t fn, float x) {
    switch (fn) {
    case EXT_SQ: return f_sq(x);
    case EXT_CUBE: return f_cube(x);
    case EXT_CBRT: return f_cbrt(x);
    case EXT_TANH: return f_tanh(x);
    case EXT_ATAN: return f_atan(x);
    case EXT_SINH: return f_sinh(x);
    default: return f_cosh(x);
    }
}

}  // namespace

// shared memory of one block: the program's words, then per warp the tape
// [CAP words][RPT rows][32 lanes] and the adjoint slots [NSLOT][RPT][32]
template <int RPT, int WARPS, int CAP, int NSLOT>
constexpr size_t grad_smem_bytes() {
    return ((size_t)(CAP + 2) * sizeof(uint2) + 15) / 16 * 16 +
           (size_t)WARPS * (CAP + NSLOT) * RPT * 32 * sizeof(float);
}

template <int RPT, int WARPS, int CAP, int NSLOT, int MINB, bool XREG>
__global__ void __launch_bounds__(WARPS * 32, MINB) grad_kernel(const GradArgs a) {
    extern __shared__ float4 smem_grad[];
    uint2 *cbuf = reinterpret_cast<uint2 *>(smem_grad);
    float *tape_all = reinterpret_cast<float *>(smem_grad + ((CAP + 2) * sizeof(uint2) + 15) / 16);
    float *slot_all = tape_all + (size_t)WARPS * CAP * RPT * 32;
    __shared__ float wsum[WARPS];
    __shared__ float wgrad[WARPS][GP_MAX_CONSTS];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // element (word i, row j) of this lane: tape[(i * RPT + j) * 32]
    float *tape = tape_all + (size_t)warp * CAP * RPT * 32 + lane;
    float *adjs = slot_all + (size_t)warp * NSLOT * RPT * 32 + lane;
    int cls_begin = 0;
    for (int b = 0; b < a.bucket; ++b) cls_begin += a.class_count[b];
    const int n_cls = a.class_count[a.bucket];
    const unsigned long long total = (unsigned long long)n_cls * (unsigned long long)a.n_chunks;
    const bool two_feat = XREG && a.n_feat == 2;

    for (unsigned long long it = 0; it <= total; ++it) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter + a.bucket, 1ULL);
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
        float *gp = a.gpart + ((size_t)p * a.n_chunks + chunk) * GP_MAX_CONSTS;
        if (m.status != GP_PROG_OK || m.n_consts > GP_MAX_CONSTS || m.n_ins > CAP) {
            if (threadIdx.x == 0) {
                a.part[(size_t)p * a.n_chunks + chunk] = __int_as_float(0x7fc00000);
                if (m.n_consts > GP_MAX_CONSTS) atomicOr(a.dev_status, GP_DEV_TOO_MANY_CONSTS);
            }
            if (threadIdx.x < GP_MAX_CONSTS) gp[threadIdx.x] = __int_as_float(0x7fc00000);
            __syncthreads();  // s_item is rewritten at the top
            continue;
        }
        const int n_ins = m.n_ins;
        for (int i = threadIdx.x; i < n_ins; i += WARPS * 32) cbuf[i] = a.code[(size_t)p * kCodeStride + i];
        __syncthreads();

        const int64_t rb = (int64_t)chunk * a.chunk_rows;
        const int64_t re = min(a.n_rows, rb + a.chunk_rows);
        const int n_in = (int)(re - rb);
        float gs[GP_MAX_CONSTS];
#pragma unroll
        for (int k = 0; k < GP_MAX_CONSTS; ++k) gs[k] = 0.0f;
        float ls = 0.0f, lc = 0.0f;
        for (int base = warp * 32 * RPT; base < n_in; base += WARPS * 32 * RPT) {
            const int o = base + lane * RPT;
            const bool full = __all_sync(0xffffffffu, o + RPT <= n_in);
            const int nv = full ? RPT : n_in - o;
            const int64_t r0 = rb + o;
            float x0[RPT], x1[RPT];
            if (XREG) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    x0[j] = (j < nv) ? __ldg(a.X + r0 + j) : 0.0f;
                    x1[j] = two_feat ? ((j < nv) ? __ldg(a.X + a.ld + r0 + j) : 0.0f) : x0[j];
                }
            }
            // the value of column feat on the lane's rows
            auto column = [&](uint32_t feat, float (&u)[RPT]) {
                if (XREG) {
#pragma unroll
                    for (int j = 0; j < RPT; ++j) u[j] = feat ? x1[j] : x0[j];
                } else {
#pragma unroll
                    for (int j = 0; j < RPT; ++j)
                        u[j] = (j < nv) ? __ldg(a.X + (int64_t)feat * a.ld + r0 + j) : 0.0f;
                }
            };
            // ---- forward: every word's result onto the tape (one switch
            // per word over its operation, each case with its operands)
            float t[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) t[j] = 0.0f;
            for (int i = 0; i < n_ins - 1; ++i) {
                const uint2 ins = cbuf[i];
                const uint32_t w = __shfl_sync(0xffffffffu, ins.x, 0);
                const float c = __uint_as_float(ins.y);
                float u[RPT];
#define GP_TAPE(q) tape[((q) * RPT + j) * 32]
#define GP_ROWS(stmt) _Pragma("unroll") for (int j = 0; j < RPT; ++j) { stmt; }
                switch (w & 31u) {
                case OP_PUSH_X: case OP_PUSH_X_SP: column(w >> 16, u); GP_ROWS(t[j] = u[j]) break;
                case OP_PUSH_C: case OP_PUSH_C_SP: GP_ROWS(t[j] = c) break;
                case OP_ADD_S: GP_ROWS(t[j] = f_add(t[j], GP_TAPE(w >> 24))) break;
                case OP_SUB_S: GP_ROWS(t[j] = f_sub(t[j], GP_TAPE(w >> 24))) break;
                case OP_MUL_S: GP_ROWS(t[j] = f_mul(t[j], GP_TAPE(w >> 24))) break;
                case OP_DIV_S: GP_ROWS(t[j] = f_div(t[j], GP_TAPE(w >> 24))) break;
                case OP_ADD_X: column(w >> 16, u); GP_ROWS(t[j] = f_add(t[j], u[j])) break;
                case OP_ADD_C: GP_ROWS(t[j] = f_add(t[j], c)) break;
                case OP_SUB_X: column(w >> 16, u); GP_ROWS(t[j] = f_sub(t[j], u[j])) break;
                case OP_SUB_C: GP_ROWS(t[j] = f_sub(t[j], c)) break;
                case OP_RSUB_X: column(w >> 16, u); GP_ROWS(t[j] = f_sub(u[j], t[j])) break;
                case OP_RSUB_C: GP_ROWS(t[j] = f_sub(c, t[j])) break;
                case OP_MUL_X: column(w >> 16, u); GP_ROWS(t[j] = f_mul(t[j], u[j])) break;
                case OP_MUL_C: GP_ROWS(t[j] = f_mul(t[j], c)) break;
                case OP_DIV_X: column(w >> 16, u); GP_ROWS(t[j] = f_div(t[j], u[j])) break;
                case OP_DIV_C: GP_ROWS(t[j] = f_div(t[j], c)) break;
                case OP_RDIV_X: column(w >> 16, u); GP_ROWS(t[j] = f_div(u[j], t[j])) break;
                case OP_RDIV_C: GP_ROWS(t[j] = f_div(c, t[j])) break;
                case OP_SQRT: GP_ROWS(t[j] = f_sqrt(t[j])) break;
                case OP_LOG: GP_ROWS(t[j] = f_log(t[j])) break;
                case OP_EXP: GP_ROWS(t[j] = f_exp(t[j])) break;
                case OP_SIN: case OP_COS: case OP_TAN: trig_rows<RPT>(t, (int)((w & 31u) - OP_SIN)); break;
                case OP_ABS: GP_ROWS(t[j] = f_abs(t[j])) break;
                case OP_NEG: GP_ROWS(t[j] = f_neg(t[j])) break;
                case OP_INV: GP_ROWS(t[j] = f_inv(t[j])) break;
                case OP_EXT1: GP_ROWS(t[j] = f_ext1((w >> 16) & 7u, t[j])) break;
                case OP_EXT2:
                    if (((w >> 16) & 7u) == EXT_MAX) { GP_ROWS(t[j] = f_max(t[j], GP_TAPE(w >> 24))) }
                    else { GP_ROWS(t[j] = f_min(t[j], GP_TAPE(w >> 24))) }
                    break;
                default: break;  // OP_END is never reached here
                }
                GP_ROWS(GP_TAPE(i) = t[j])
            }
            // ---- the loss and its derivative per row
            float at[RPT];
            {
                float e = 0.0f;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const bool in = j < nv;
                    const float yv = in ? __ldg(a.y + r0 + j) : 0.0f;
                    const float wv = (a.w && in) ? __ldg(a.w + r0 + j) : 1.0f;
                    float l = row_loss(a.metric, t[j], yv);
                    if (a.w) l = __fmul_rn(wv, l);
                    e = in ? __fadd_rn(e, l) : e;
                    at[j] = in ? __fmul_rn(wv, g_dloss(a.metric, t[j], yv)) : 0.0f;
                }
                kahan_add(ls, lc, e);
            }
            // the lane's share of constant k: its rows' adjoints times d
#define GP_SHARE(k, d)                                                     \
    {                                                                      \
        float s_ = 0.0f;                                                   \
        _Pragma("unroll") for (int j = 0; j < RPT; ++j)                    \
            s_ = (j < nv) ? __fadd_rn(s_, __fmul_rn(at[j], (d))) : s_;     \
        gadd(gs, (k), s_);                                                 \
    }
            // ---- adjoint: the words in reverse, one switch per word; the
            // word's input is the previous word's result (tin), its output
            // its own (v); a popped slot's value is the spilled word's result
            for (int i = n_ins - 2; i >= 0; --i) {
                const uint2 ins = cbuf[i];
                const uint32_t w = __shfl_sync(0xffffffffu, ins.x, 0);
                const float c = __uint_as_float(ins.y);
                const uint32_t slot = min((w >> 8) & 255u, (uint32_t)NSLOT - 1u);
                const uint32_t aux = w >> 24;
#define GP_ADJ(j) adjs[(slot * RPT + (j)) * 32]
#define GP_TIN GP_TAPE(i - 1)
#define GP_V GP_TAPE(i)
                float u[RPT];
                switch (w & 31u) {
                case OP_PUSH_X: break;
                case OP_PUSH_X_SP: GP_ROWS(at[j] = GP_ADJ(j)) break;
                case OP_PUSH_C: GP_SHARE(aux, 1.0f) break;
                case OP_PUSH_C_SP: GP_SHARE(aux, 1.0f) GP_ROWS(at[j] = GP_ADJ(j)) break;
                case OP_ADD_S: GP_ROWS(GP_ADJ(j) = at[j]) break;
                case OP_SUB_S: GP_ROWS(GP_ADJ(j) = -at[j]) break;
                case OP_MUL_S:
                    GP_ROWS(GP_ADJ(j) = __fmul_rn(at[j], GP_TIN); at[j] = __fmul_rn(at[j], GP_TAPE(aux)))
                    break;
                case OP_DIV_S:
                    GP_ROWS(const float r = GP_TAPE(aux); const bool p0 = fabsf(r) < kThr;
                            GP_ADJ(j) = p0 ? 0.0f : __fmul_rn(at[j], -__fdiv_rn(GP_V, r));
                            at[j] = p0 ? 0.0f : __fmul_rn(at[j], __frcp_rn(r)))
                    break;
                case OP_ADD_X: case OP_SUB_X: break;
                case OP_ADD_C: GP_SHARE(aux, 1.0f) break;
                case OP_SUB_C: GP_SHARE(aux, -1.0f) break;
                case OP_RSUB_X: GP_ROWS(at[j] = -at[j]) break;
                case OP_RSUB_C: GP_SHARE(aux, 1.0f) GP_ROWS(at[j] = -at[j]) break;
                case OP_MUL_X: column(w >> 16, u); GP_ROWS(at[j] = __fmul_rn(at[j], u[j])) break;
                case OP_MUL_C: GP_SHARE(aux, GP_TIN) GP_ROWS(at[j] = __fmul_rn(at[j], c)) break;
                case OP_DIV_X:
                    column(w >> 16, u);
                    GP_ROWS(at[j] = fabsf(u[j]) < kThr ? 0.0f : __fmul_rn(at[j], __frcp_rn(u[j])))
                    break;
                case OP_DIV_C:
                    if (fabsf(c) < kThr) { GP_ROWS(at[j] = 0.0f) }
                    else {
                        GP_SHARE(aux, -__fdiv_rn(GP_V, c))
                        GP_ROWS(at[j] = __fmul_rn(at[j], __frcp_rn(c)))
                    }
                    break;
                case OP_RDIV_X:
                    GP_ROWS(const float r = GP_TIN;
                            at[j] = fabsf(r) < kThr ? 0.0f : __fmul_rn(at[j], -__fdiv_rn(GP_V, r)))
                    break;
                case OP_RDIV_C:
                    GP_SHARE(aux, fabsf(GP_TIN) < kThr ? 0.0f : __frcp_rn(GP_TIN))
                    GP_ROWS(const float r = GP_TIN;
                            at[j] = fabsf(r) < kThr ? 0.0f : __fmul_rn(at[j], -__fdiv_rn(GP_V, r)))
                    break;
                case OP_EXT2:
                    GP_ROWS(const float l = GP_TIN; const float r = GP_TAPE(aux);
                            const bool left = (((w >> 16) & 7u) == EXT_MAX) ? (l > r || l != l)
                                                                             : (l < r || l != l);
                            GP_ADJ(j) = left ? 0.0f : at[j]; at[j] = left ? at[j] : 0.0f)
                    break;
                default:  // the unary functions
                    GP_ROWS(at[j] = __fmul_rn(at[j], d_unary(w & 31u, (w >> 16) & 7u, GP_TIN, GP_V)))
                    break;
                }
#undef GP_ADJ
#undef GP_TIN
#undef GP_V
            }
#undef GP_SHARE
#undef GP_ROWS
#undef GP_TAPE
        }
        // fixed butterfly per warp, then the warps in order
        float lv = __fsub_rn(ls, lc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lv = __fadd_rn(lv, __shfl_xor_sync(0xffffffffu, lv, off));
        if (lane == 0) wsum[warp] = lv;
#pragma unroll
        for (int k = 0; k < GP_MAX_CONSTS; ++k) {
            float v = gs[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
            if (lane == 0) wgrad[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float v = 0.0f;
            for (int q = 0; q < WARPS; ++q) v = __fadd_rn(v, wsum[q]);
            a.part[(size_t)p * a.n_chunks + chunk] = v;
        } else if (threadIdx.x >= 32 && threadIdx.x < 32 + GP_MAX_CONSTS) {
            const int k = threadIdx.x - 32;
            float v = 0.0f;
            for (int q = 0; q < WARPS; ++q) v = __fadd_rn(v, wgrad[q][k]);
            gp[k] = v;
        }
        __syncthreads();  // wsum, wgrad, cbuf and s_item are reused
    }
}

template <int RPT, int WARPS, int CAP, int NSLOT, int MINB, bool XREG>
cudaError_t launch_grad_t(const GradArgs &a, int sms, cudaStream_t st, int *occ_out) {
    constexpr size_t smem = grad_smem_bytes<RPT, WARPS, CAP, NSLOT>();
    auto k = grad_kernel<RPT, WARPS, CAP, NSLOT, MINB, XREG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ_out) {
        *occ_out = occ;
        return cudaSuccess;
    }
    k<<<sms * (occ > 0 ? occ : 1), WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// One row per lane (a tape row per word per lane; two rows per lane halved
// the resident warps and ran 33% slower).  Buckets 0-3 (compiled depth <=
// 8, 7 adjoint slots): 8, 8, 8 and 4 warps per block, as many blocks as
// the tape and registers allow; bucket 4 (up to 256 words or deeper
// stacks): 2 warps and 19 slots.
#define GP_GRAD_LAUNCH(R, W, C, S, M) \
    (xreg ? launch_grad_t<R, W, C, S, M, true>(a, sms, st, occ) \
          : launch_grad_t<R, W, C, S, M, false>(a, sms, st, occ))
cudaError_t launch_grad(const GradArgs &a, int sms, cudaStream_t st, int *occ) {
    const bool xreg = a.n_feat <= 2;
    switch (a.bucket) {
    case 0: return GP_GRAD_LAUNCH(1, 8, kGradCap0, kSmallDepth - 1, 5);
    case 1: return GP_GRAD_LAUNCH(1, 8, kGradCap1, kSmallDepth - 1, 4);
    case 2: return GP_GRAD_LAUNCH(1, 8, kGradCap2, kSmallDepth - 1, 2);
    case 3: return GP_GRAD_LAUNCH(1, 4, kGradCap3, kSmallDepth - 1, 2);
    default: return GP_GRAD_LAUNCH(1, 2, kCodeStride, kDeepSlots, 3);
    }
}
#undef GP_GRAD_LAUNCH

// Adam: one thread per program walks its prefix list; the k-th CONST node
// takes slot k of grad / m / v.
__global__ void __launch_bounds__(128) adam_kernel(AdamArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_progs) return;
    const int off = a.offsets[p];
    const int len = a.offsets[p + 1] - off;
    if (len < 1 || len > GP_MAX_LEN) return;
    const float b1t = 1.0f - powf(a.beta1, (float)a.step);
    const float b2t = 1.0f - powf(a.beta2, (float)a.step);
    int k = 0;
    for (int j = 0; j < len && k < GP_MAX_CONSTS; ++j) {
        gp_node *nd = a.progs + off + j;
        if (nd->op != GP_CONST) continue;
        const size_t i = (size_t)p * GP_MAX_CONSTS + k;
        const float g = a.grad[i];
        if (isfinite(g)) {
            const float mi = __fadd_rn(__fmul_rn(a.beta1, a.m[i]), __fmul_rn(1.0f - a.beta1, g));
            const float vi = __fadd_rn(__fmul_rn(a.beta2, a.v[i]),
                                       __fmul_rn(1.0f - a.beta2, __fmul_rn(g, g)));
            a.m[i] = mi;
            a.v[i] = vi;
            const float mh = __fdiv_rn(mi, b1t);
            const float vh = __fdiv_rn(vi, b2t);
            const float stp = __fdiv_rn(__fmul_rn(a.lr, mh), __fadd_rn(__fsqrt_rn(vh), a.eps));
            nd->c = __fsub_rn(nd->c, stp);
        }
        ++k;
    }
}

cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st) {
    if (a.n_progs <= 0) return cudaSuccess;
    adam_kernel<<<(a.n_progs + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// One thread per program: the k-th CONST node in prefix order is slot k.
__global__ void __launch_bounds__(128) consts_kernel(gp_node *progs, const int32_t *offsets,
                                                     int n_progs, float *consts, bool to_nodes) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_progs) return;
    const int off = offsets[p];
    const int len = offsets[p + 1] - off;
    float *row = consts + (size_t)p * GP_MAX_CONSTS;
    int k = 0;
    if (len >= 1 && len <= GP_MAX_LEN) {
        for (int j = 0; j < len && k < GP_MAX_CONSTS; ++j) {
            gp_node *nd = progs + off + j;
            if (nd->op != GP_CONST) continue;
            if (to_nodes) nd->c = row[k];
            else row[k] = nd->c;
            ++k;
        }
    }
    if (!to_nodes)
        for (; k < GP_MAX_CONSTS; ++k) row[k] = 0.0f;
}

cudaError_t launch_consts(gp_node *progs, const int32_t *offsets, int n_progs, float *consts,
                          bool to_nodes, cudaStream_t st) {
    if (n_progs <= 0) return cudaSuccess;
    consts_kernel<<<(n_progs + 127) / 128, 128, 0, st>>>(progs, offsets, n_progs, consts, to_nodes);
    return cudaGetLastError();
}

}  // namespace gpk
