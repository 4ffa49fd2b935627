// gp_grad.cu -- gradients of fitness with respect to the ephemeral
// constants (forward mode), and one Adam step on the constants.  Neither
// has a counterpart in the paper; they serve constant tuning between
// generations.
//
// Forward mode on the compiled stack form of the evaluator
// (gp_internal.cuh), in its gradient variant: no constant-only subtree is
// folded, and a marker word precedes every word whose operands hold
// constants, naming the constants under each operand (they form contiguous
// ranges of the prefix-order numbering).  Each row carries one tangent per
// constant, dt[k] = d(value holding c_k)/d(c_k): a pushed constant starts
// at 1, and a marked word multiplies the tangents under each operand by
// its partial derivative with respect to that operand, so after the root
// dt[k] is d(program)/d(c_k).  Every constant is a leaf used once, so a
// row costs the forward pass plus one multiply per (constant, ancestor)
// pair -- no tape and no reverse sweep: the values and tangents live in
// registers and a few shared-memory slots per row.
//
// A block takes one (program, row chunk) item; its warps run the program
// over their own sub-tiles of 128 rows (4 per lane) with the evaluator's
// fast loop (the same FP32 operations, so the fitness equals
// gp_evaluate's), which hands each marked word back to grad_word.  The
// loss derivative per row times the tangents gives each constant's share.
// Programs are bucketed by their number of constants (the tangent slots
// per row) and stack depth, one launch per bucket.  Per-lane sums are FP32
// (the loss Kahan-compensated), warp sums fixed-order, chunk sums FP64 in
// order (gp_reduce.cu).
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

// The tangents of a lane's four rows: one float4 per constant k at the
// shared-memory address db + k * 512.  They are read and written only by
// volatile asm statements (here and in the fast loop, which declares no
// memory clobber), so their order is kept.
__device__ __forceinline__ float4 tan_load(uint32_t a) {
    float4 d;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(d.x), "=f"(d.y), "=f"(d.z), "=f"(d.w)
                 : "r"(a));
    return d;
}
__device__ __forceinline__ void tan_store(uint32_t a, float4 d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(d.x), "f"(d.y),
                 "f"(d.z), "f"(d.w)
                 : "memory");
}

// One word of the gradient form that the fast loop handed back (a marked
// word it does not run or whose fast path gave up, or an unmarked word it
// does not run): its value with the evaluator's operations and, after a
// marker (mk != 0), its partial derivatives with respect to the top
// operand t (pt) and the other operand (po), applied to the tangents of
// the constants under each (kGradMark).  Four rows per lane; the stack
// slot of this lane's rows is one float4 (sb + slot * 512 bytes), the
// tangent of constant k one float4 at db + k * 512.
template <int NSLOT, int KT, bool XREG>
__device__ __forceinline__ void grad_word(uint32_t w, float c, uint32_t mk, float (&t)[4],
                                          const float (&x0)[4], const float (&x1)[4],
                                          const float *__restrict__ X, int64_t ld, int64_t r0,
                                          int64_t re, bool vec, uint32_t sb, uint32_t db) {
    constexpr int R = 4;
    const uint32_t op = w & 31u;
    const uint32_t fn = (w >> 16) & 7u;
    const uint32_t sa = sb + min((w >> 8) & 255u, (uint32_t)NSLOT - 1u) * 32u * 16u;
    // the other operand: a stack slot (S forms, EXT2), a column (X forms,
    // PUSH_X), else the word's constant
    float o[R];
    const bool from_slot = (op >= OP_ADD_S && op <= OP_DIV_S) || op == OP_EXT2;
    const bool from_col = op == OP_PUSH_X || op == OP_PUSH_X_SP ||
                          (op >= OP_ADD_X && op <= OP_RDIV_X && ((op - OP_ADD_X) & 1u) == 0u);
    if (from_slot) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3])
                     : "r"(sa));
    } else if (from_col) {
        const int feat = (int)(w >> 16);
        if (XREG) {
#pragma unroll
            for (int j = 0; j < R; ++j) o[j] = feat ? x1[j] : x0[j];
        } else {
            load_rows<R>(o, X + (int64_t)feat * ld, r0, re, vec);
        }
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) o[j] = c;
    }
    if (op == OP_PUSH_X_SP || op == OP_PUSH_C_SP)
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(sa), "f"(t[0]), "f"(t[1]),
                     "f"(t[2]), "f"(t[3])
                     : "memory");
    float v[R];
#define GP_ROWS(stmt) _Pragma("unroll") for (int j = 0; j < R; ++j) { stmt; }
    switch (op) {
    case OP_ADD_S: case OP_ADD_X: case OP_ADD_C: GP_ROWS(v[j] = f_add(t[j], o[j])) break;
    case OP_SUB_S: case OP_SUB_X: case OP_SUB_C: GP_ROWS(v[j] = f_sub(t[j], o[j])) break;
    case OP_RSUB_X: case OP_RSUB_C: GP_ROWS(v[j] = f_sub(o[j], t[j])) break;
    case OP_MUL_S: case OP_MUL_X: case OP_MUL_C: GP_ROWS(v[j] = f_mul(t[j], o[j])) break;
    case OP_DIV_S: case OP_DIV_X: case OP_DIV_C: GP_ROWS(v[j] = f_div(t[j], o[j])) break;
    case OP_RDIV_X: case OP_RDIV_C: GP_ROWS(v[j] = f_div(o[j], t[j])) break;
    case OP_SQRT: GP_ROWS(v[j] = f_sqrt(t[j])) break;
    case OP_LOG: GP_ROWS(v[j] = f_log(t[j])) break;
    case OP_EXP: GP_ROWS(v[j] = f_exp(t[j])) break;
    case OP_SIN: case OP_COS: case OP_TAN:
        GP_ROWS(v[j] = t[j])
        trig_rows<R>(v, (int)(op - OP_SIN));
        break;
    case OP_ABS: GP_ROWS(v[j] = f_abs(t[j])) break;
    case OP_NEG: GP_ROWS(v[j] = f_neg(t[j])) break;
    case OP_INV: GP_ROWS(v[j] = f_inv(t[j])) break;
    case OP_EXT1: GP_ROWS(v[j] = f_ext1(fn, t[j])) break;
    case OP_EXT2:
        if (fn == EXT_MAX) { GP_ROWS(v[j] = f_max(t[j], o[j])) }
        else { GP_ROWS(v[j] = f_min(t[j], o[j])) }
        break;
    default: GP_ROWS(v[j] = o[j]) break;  // the pushes (OP_END never gets here)
    }
    if (mk != 0u) {
        float pt[R], po[R];
        GP_ROWS(pt[j] = 1.0f; po[j] = 1.0f)
        switch (op) {
        case OP_SUB_S: case OP_SUB_X: case OP_SUB_C: GP_ROWS(po[j] = -1.0f) break;
        case OP_RSUB_X: case OP_RSUB_C: GP_ROWS(pt[j] = -1.0f) break;
        case OP_MUL_S: case OP_MUL_X: case OP_MUL_C: GP_ROWS(pt[j] = o[j]; po[j] = t[j]) break;
        case OP_DIV_S: case OP_DIV_X: case OP_DIV_C:
            GP_ROWS(const bool p0 = fabsf(o[j]) < kThr;
                    pt[j] = p0 ? 0.0f : __frcp_rn(o[j]);
                    po[j] = p0 ? 0.0f : -__fdiv_rn(v[j], o[j]))
            break;
        case OP_RDIV_X: case OP_RDIV_C:
            GP_ROWS(const bool p0 = fabsf(t[j]) < kThr;
                    pt[j] = p0 ? 0.0f : -__fdiv_rn(v[j], t[j]);
                    po[j] = p0 ? 0.0f : __frcp_rn(t[j]))
            break;
        case OP_EXT2:
            GP_ROWS(const bool left = (fn == EXT_MAX) ? (t[j] > o[j] || t[j] != t[j])
                                                      : (t[j] < o[j] || t[j] != t[j]);
                    pt[j] = left ? 1.0f : 0.0f; po[j] = left ? 0.0f : 1.0f)
            break;
        case OP_SQRT: case OP_LOG: case OP_EXP: case OP_SIN: case OP_COS: case OP_TAN:
        case OP_ABS: case OP_NEG: case OP_INV: case OP_EXT1:
            GP_ROWS(pt[j] = d_unary(op, fn, t[j], v[j]))
            break;
        default: break;  // add and the pushes: both partials 1
        }
        const int tlo = (int)(mk & 31u), thi = min((int)((mk >> 5) & 31u), KT);
        const int olo = (int)((mk >> 10) & 31u), ohi = min((int)((mk >> 15) & 31u), KT);
        const bool fresh = ((mk >> 20) & 1u) != 0u;
        for (int k = tlo; k < thi; ++k) {
            float4 d = tan_load(db + (uint32_t)k * 512u);
            d.x = __fmul_rn(d.x, pt[0]);
            d.y = __fmul_rn(d.y, pt[1]);
            d.z = __fmul_rn(d.z, pt[2]);
            d.w = __fmul_rn(d.w, pt[3]);
            tan_store(db + (uint32_t)k * 512u, d);
        }
        for (int k = olo; k < ohi; ++k) {
            float4 d = fresh ? make_float4(1.0f, 1.0f, 1.0f, 1.0f) : tan_load(db + (uint32_t)k * 512u);
            d.x = __fmul_rn(d.x, po[0]);
            d.y = __fmul_rn(d.y, po[1]);
            d.z = __fmul_rn(d.z, po[2]);
            d.w = __fmul_rn(d.w, po[3]);
            tan_store(db + (uint32_t)k * 512u, d);
        }
    }
    GP_ROWS(t[j] = v[j])
#undef GP_ROWS
}

// Runs one program of the gradient form over the lane's four rows: the
// gradient variant of the fast loop runs the words it can, marked ones
// with their tangent updates, and each word it hands back -- a marker with
// the word after it, or a word it does not run -- runs in grad_word.
// Returns the prediction in t and leaves each constant's tangent
// d(prediction)/d(c_k) at db + k * 512.
template <int NSLOT, int KT, bool XREG>
__device__ __forceinline__ void grad_run(float (&t)[4], const uint2 *cbuf, const float (&x0)[4],
                                         const float (&x1)[4], const float *__restrict__ X,
                                         int64_t ld, int64_t r0, int64_t re, bool vec,
                                         float4 *stk, uint32_t db) {
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = 0.0f;
    uint32_t pa = (uint32_t)__cvta_generic_to_shared(cbuf);
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(stk);
    const uint64_t x0p[2] = {pack2(x0[0], x0[1]), pack2(x0[2], x0[3])};
    const uint64_t x1p[2] = {pack2(x1[0], x1[1]), pack2(x1[2], x1[3])};
#pragma unroll 1
    for (;;) {
        uint64_t tp[2] = {pack2(t[0], t[1]), pack2(t[2], t[3])};
        uint32_t hw;
        float hc;
        if constexpr (XREG) fast_r4_divs_x_grad<NSLOT, KT>(pa, tp, x0p, x1p, sb, db, hw, hc);
        else fast_r4_divs_nox_grad<NSLOT, KT>(pa, tp, x0p, x1p, sb, db, hw, hc);
        unpack2(tp[0], t[0], t[1]);
        unpack2(tp[1], t[2], t[3]);
        uint32_t w = __shfl_sync(0xffffffffu, hw, 0);
        float c = hc;
        uint32_t mk = 0u;
        if ((w & 63u) == kGradMark) {
            mk = __shfl_sync(0xffffffffu, __float_as_uint(hc), 0);
            uint32_t w2, c2;
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(w2), "=r"(c2) : "r"(pa));
            pa += 8u;
            w = __shfl_sync(0xffffffffu, w2, 0);
            c = __uint_as_float(c2);
        }
        if ((w & 31u) == OP_END) break;
        grad_word<NSLOT, KT, XREG>(w, c, mk, t, x0, x1, X, ld, r0, re, vec, sb, db);
    }
}

// shared memory of one block: the program's words (through the buffer's
// end OP_END), then per warp the value stack [NSLOT][32 lanes] and the
// tangents [KT][32 lanes], one float4 (four rows) per entry
template <int WARPS, int NSLOT, int KT>
constexpr size_t grad_smem_bytes() {
    return (size_t)(kGradCodeStride + 2) * sizeof(uint2) +
           (size_t)WARPS * (NSLOT + KT) * 32 * sizeof(float4);
}

template <int WARPS, int NSLOT, int KT, int MINB, bool XREG>
__global__ void __launch_bounds__(WARPS * 32, MINB) grad_kernel(const GradArgs a) {
    constexpr int R = 4;
    static_assert((kGradCodeStride + 2) * sizeof(uint2) % 16 == 0, "stack alignment");
    extern __shared__ float4 smem_grad[];
    uint2 *cbuf = reinterpret_cast<uint2 *>(smem_grad);
    float4 *stack_all = smem_grad + (kGradCodeStride + 2) * sizeof(uint2) / 16;
    float4 *tan_all = stack_all + (size_t)WARPS * NSLOT * 32;
    __shared__ float wsum[WARPS];
    __shared__ float wgrad[WARPS][GP_MAX_CONSTS];
    __shared__ unsigned long long s_item;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4 *stk = stack_all + (size_t)warp * NSLOT * 32 + lane;
    const uint32_t db = (uint32_t)__cvta_generic_to_shared(tan_all + (size_t)warp * KT * 32 + lane);
    int cls_begin = 0;
    for (int b = 0; b < a.bucket; ++b) cls_begin += a.class_count[b];
    const int n_cls = a.class_count[a.bucket];
    const unsigned long long total = (unsigned long long)n_cls * (unsigned long long)a.n_chunks;
    const bool vec = a.vec_ok != 0;
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
        if (m.status != GP_PROG_OK || m.n_consts > KT || m.n_ins > kGradCodeStride) {
            if (threadIdx.x == 0) {
                a.part[(size_t)p * a.n_chunks + chunk] = __int_as_float(0x7fc00000);
                if (m.n_consts > GP_MAX_CONSTS) atomicOr(a.dev_status, GP_DEV_TOO_MANY_CONSTS);
            }
            if (threadIdx.x < GP_MAX_CONSTS) gp[threadIdx.x] = __int_as_float(0x7fc00000);
            __syncthreads();  // s_item is rewritten at the top
            continue;
        }
        const int n_ins = m.n_ins;
        const uint2 *src = a.code + (size_t)p * kGradCodeStride;
        for (int i = threadIdx.x; i < kGradCodeStride + 2; i += WARPS * 32)
            cbuf[i] = (i < n_ins) ? src[i] : make_uint2(make_ins(OP_END, 0, 0), 0u);
        __syncthreads();

        const int nc = m.n_consts;
        const int64_t rb = (int64_t)chunk * a.chunk_rows;
        const int64_t re = min(a.n_rows, rb + a.chunk_rows);
        const int n_in = (int)(re - rb);
        float gs[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) gs[k] = 0.0f;
        float ls = 0.0f, lc = 0.0f;
        for (int base = warp * 32 * R; base < n_in; base += WARPS * 32 * R) {
            const int o = base + lane * R;
            const bool full = __all_sync(0xffffffffu, o + R <= n_in);
            const int nv = full ? R : n_in - o;
            float x0[R], x1[R];
            if (XREG) {
                load_chunk_rows<R>(x0, a.X + (rb + o), full && vec, nv);
                if (two_feat) load_chunk_rows<R>(x1, a.X + (a.ld + rb + o), full && vec, nv);
                else {
#pragma unroll
                    for (int j = 0; j < R; ++j) x1[j] = x0[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) x0[j] = x1[j] = 0.0f;
            }
            float t[R];
            grad_run<NSLOT, KT, XREG>(t, cbuf, x0, x1, a.X, a.ld, rb + o, re, vec, stk, db);
            // the loss and its derivative per row
            float yv[R], wv[R];
            load_chunk_rows<R>(yv, a.y + (rb + o), full && vec, nv);
            if (a.w) load_chunk_rows<R>(wv, a.w + (rb + o), full && vec, nv);
            else {
#pragma unroll
                for (int j = 0; j < R; ++j) wv[j] = 1.0f;
            }
            float e = 0.0f, at[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const bool in = j < nv;
                float l = row_loss(a.metric, t[j], yv[j]);
                if (a.w) l = __fmul_rn(wv[j], l);
                e = in ? __fadd_rn(e, l) : e;
                at[j] = in ? __fmul_rn(wv[j], g_dloss(a.metric, t[j], yv[j])) : 0.0f;
            }
            kahan_add(ls, lc, e);
            // each constant's share: the rows' loss derivatives times its tangents
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                if (k < nc) {
                    const float4 d = tan_load(db + (uint32_t)k * 512u);
                    const float dd[R] = {d.x, d.y, d.z, d.w};
                    float s = 0.0f;
#pragma unroll
                    for (int j = 0; j < R; ++j) s = (j < nv) ? __fadd_rn(s, __fmul_rn(at[j], dd[j])) : s;
                    gs[k] = __fadd_rn(gs[k], s);
                }
            }
        }
        // fixed butterfly per warp, then the warps in order
        float lv = __fsub_rn(ls, lc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lv = __fadd_rn(lv, __shfl_xor_sync(0xffffffffu, lv, off));
        if (lane == 0) wsum[warp] = lv;
#pragma unroll
        for (int k = 0; k < GP_MAX_CONSTS; ++k) {
            float v = 0.0f;
            if (k < KT) {
                v = gs[k < KT ? k : 0];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
            }
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

template <int WARPS, int NSLOT, int KT, int MINB, bool XREG>
cudaError_t launch_grad_t(const GradArgs &a, int sms, cudaStream_t st, int *occ_out) {
    constexpr size_t smem = grad_smem_bytes<WARPS, NSLOT, KT>();
    auto k = grad_kernel<WARPS, NSLOT, KT, MINB, XREG>;
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

// Four rows per lane.  Buckets 0-2 (compiled depth <= 8, 7 stack slots):
// 8 warps with 4, 8 or 16 tangent slots per row, 4, 3 or 2 blocks per SM
// (shared memory allows no more); bucket 3 (deeper stacks): 4 warps, 19
// slots, 3 blocks.
#define GP_GRAD_LAUNCH(W, S, K, M) \
    (xreg ? launch_grad_t<W, S, K, M, true>(a, sms, st, occ) \
          : launch_grad_t<W, S, K, M, false>(a, sms, st, occ))
cudaError_t launch_grad(const GradArgs &a, int sms, cudaStream_t st, int *occ) {
    const bool xreg = a.n_feat <= 2;
    switch (a.bucket) {
    case 0: return GP_GRAD_LAUNCH(8, kSmallDepth - 1, kGradTan0, 4);
    case 1: return GP_GRAD_LAUNCH(8, kSmallDepth - 1, kGradTan1, 3);
    case 2: return GP_GRAD_LAUNCH(8, kSmallDepth - 1, GP_MAX_CONSTS, 2);
    default: return GP_GRAD_LAUNCH(4, kDeepSlots, GP_MAX_CONSTS, 3);
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
