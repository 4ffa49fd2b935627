// gp_compile.cu -- device pre-pass: validate each prefix list, compile it
// to the register-stack form (gp_internal.cuh), and sort the programs into
// classes (stack depth, extended functions) and by length (length-bucketed
// work queue); plus the
// deterministic total-weight sum.
#include "gp_internal.cuh"
#include "gp_interp.cuh"

namespace gpk {

static __host__ __device__ inline int op_arity(int op) {
    if (op == GP_CONST || op == GP_VAR) return 0;
    if ((op >= GP_ADD && op <= GP_DIV) || op == GP_MAX || op == GP_MIN) return 2;
    if (op >= GP_SQRT && op <= GP_COSH) return 1;
    return -1;
}

static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int n_progs, int n_chunks, bool grad, bool moments) {
    Layout L{};
    size_t o = 0;
    size_t P = (size_t)(n_progs > 0 ? n_progs : 1);
    size_t C = (size_t)(n_chunks > 0 ? n_chunks : 1);
    L.counters = o;    o = align256(o + 8 * sizeof(unsigned long long));
    L.sumw = o;        o = align256(o + sizeof(double));
    L.sumw_part = o;   o = align256(o + kSumwBlocks * sizeof(double));
    L.code = o;        o = align256(o + P * (grad ? kGradCodeStride : kCodeStride) * sizeof(uint2));
    L.meta = o;        o = align256(o + P * sizeof(ProgMeta));
    L.order = o;       o = align256(o + P * sizeof(int32_t));
    L.class_count = o; o = align256(o + (kOrderClasses + 2) * sizeof(int32_t));
    L.part = o;        o = align256(o + P * C * sizeof(float));
    if (moments) {
        L.ystat = o;      o = align256(o + 4 * sizeof(double));
        L.ystat_part = o; o = align256(o + 2 * kSumwBlocks * sizeof(double));
        L.shift = o;      o = align256(o + P * sizeof(float));
        L.mom = o;        o = align256(o + P * C * 3 * sizeof(double));
    }
    if (grad) {
        L.gpart = o;   o = align256(o + P * C * GP_MAX_CONSTS * sizeof(float));
    }
    L.total = o;
    return L;
}

Workspace carve(void *base, const Layout &L, bool grad) {
    char *b = static_cast<char *>(base);
    Workspace w{};
    w.counters = reinterpret_cast<unsigned long long *>(b + L.counters);
    w.sumw = reinterpret_cast<double *>(b + L.sumw);
    w.sumw_part = reinterpret_cast<double *>(b + L.sumw_part);
    w.code = reinterpret_cast<uint2 *>(b + L.code);
    w.meta = reinterpret_cast<ProgMeta *>(b + L.meta);
    w.order = reinterpret_cast<int32_t *>(b + L.order);
    w.class_count = reinterpret_cast<int32_t *>(b + L.class_count);
    w.part = reinterpret_cast<float *>(b + L.part);
    if (L.mom) {
        w.ystat = reinterpret_cast<double *>(b + L.ystat);
        w.ystat_part = reinterpret_cast<double *>(b + L.ystat_part);
        w.shift = reinterpret_cast<float *>(b + L.shift);
        w.mom = reinterpret_cast<double *>(b + L.mom);
    }
    if (grad) w.gpart = reinterpret_cast<float *>(b + L.gpart);
    w.bytes = L.total;
    return w;
}

// The value of a function node whose operands are all constants, computed
// with the evaluator's own FP32 operations, so the folded constant is the
// very number the evaluator would produce on every row.
__device__ float fold_unary(int op, float a) {
    switch (op) {
        case GP_SQRT: return f_sqrt(a);
        case GP_LOG: return f_log(a);
        case GP_EXP: return f_exp(a);
        case GP_SIN:
        case GP_COS:
        case GP_TAN: {
            float t[1] = {a};
            trig_rows<1>(t, op - GP_SIN);
            return t[0];
        }
        case GP_ABS: return f_abs(a);
        case GP_NEG: return f_neg(a);
        case GP_INV: return f_inv(a);
        case GP_SQ: return f_sq(a);
        case GP_CUBE: return f_cube(a);
        case GP_CBRT: return f_cbrt(a);
        case GP_TANH: return f_tanh(a);
        case GP_ATAN: return f_atan(a);
        case GP_SINH: return f_sinh(a);
        default: return f_cosh(a);
    }
}

__device__ float fold_binary(int op, float l, float r) {
    switch (op) {
        case GP_ADD: return f_add(l, r);
        case GP_SUB: return f_sub(l, r);
        case GP_MUL: return f_mul(l, r);
        case GP_DIV: return f_div(l, r);
        case GP_MAX: return f_max(l, r);
        default: return f_min(l, r);
    }
}

// One thread per program.  Passes over at most 255 nodes held in
// per-thread local arrays: (1) reverse scan for validity, subtree sizes and
// the values of constant-only subtrees, (2) mark the inside of every
// maximal constant-only subtree as dropped (its root becomes one constant)
// and the terminal children that fold into their binary parent, (3)
// reverse scan emitting instructions.  Folding constant-only subtrees
// leaves every row's result bit-identical: the same FP32 operations run on
// the same inputs, once per program instead of once per row.
__global__ void __launch_bounds__(128) compile_kernel(CompileArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_progs) return;
    const int off = a.offsets[p];
    const int len = a.offsets[p + 1] - off;
    uint2 *out = a.code + (size_t)p * (a.grad ? kGradCodeStride : kCodeStride);
    const gp_node *prog = a.progs + off;

    uint8_t size[GP_MAX_LEN];
    // terminal: 1 = folded into its parent; binary: 0 / 1 R / 2 L folded;
    // any node: 3 = inside a constant-only subtree (dropped)
    uint8_t mode[GP_MAX_LEN];
    uint8_t kon[GP_MAX_LEN];   // 1: the node's subtree holds no variable
    float kval[GP_MAX_LEN];    // its value when kon
    int status = GP_PROG_OK;
    int sp = 0, hw = 0, n_consts = 0;

    if (len < 1 || len > GP_MAX_LEN) status = GP_PROG_BAD_LENGTH;
    // pass 1: reverse scan with a stack of subtree sizes (kept in size[])
    // and of the constant-only flags and values
    uint8_t szst[GP_MAX_LEN], kst[GP_MAX_LEN];
    float vst[GP_MAX_LEN];
    // with a.shift the scan also evaluates the program at row 0 (every
    // node's value, not only the constant-only ones)
    const bool row0 = a.shift != nullptr;
    for (int j = len - 1; j >= 0 && status == GP_PROG_OK; --j) {
        const gp_node nd = prog[j];
        const int ar = op_arity(nd.op);
        mode[j] = 0;
        if (ar < 0) { status = GP_PROG_BAD_OP; break; }
        if (nd.op == GP_VAR && (nd.feat < 0 || nd.feat >= a.n_feat)) {
            status = GP_PROG_BAD_FEATURE;
            break;
        }
        int s;
        uint8_t k;
        float v = 0.0f;
        if (ar == 0) {
            s = 1;
            n_consts += (nd.op == GP_CONST);
            k = nd.op == GP_CONST;  // (the gradient form clears k of functions below)
            v = k ? nd.c : (row0 ? a.X[(int64_t)nd.feat * a.ld] : 0.0f);
        } else if (ar == 1) {
            if (sp < 1) { status = GP_PROG_UNDERFLOW; break; }
            --sp;
            s = 1 + szst[sp];
            k = a.grad ? 0 : kst[sp];
            if (k || row0) v = fold_unary(nd.op, vst[sp]);
        } else {
            if (sp < 2) { status = GP_PROG_UNDERFLOW; break; }
            // first pop is the left operand
            const int l = szst[sp - 1], r = szst[sp - 2];
            k = a.grad ? 0 : (kst[sp - 1] & kst[sp - 2]);
            if (k || row0) v = fold_binary(nd.op, vst[sp - 1], vst[sp - 2]);
            sp -= 2;
            s = 1 + l + r;
        }
        size[j] = (uint8_t)s;
        kon[j] = k;
        kval[j] = v;
        szst[sp] = (uint8_t)s;
        kst[sp] = k;
        vst[sp] = v;
        ++sp;
        if (sp > hw) hw = sp;
    }
    if (status == GP_PROG_OK && sp != 1) status = GP_PROG_LEFTOVER;
    if (status == GP_PROG_OK && hw > GP_MAX_STACK) status = GP_PROG_TOO_DEEP;
    if (a.out_prog_status) a.out_prog_status[p] = status;
    if (row0) {
        // a non-finite value would poison every shifted row; 0 is as good
        // as any other finite shift
        const float k0 = (status == GP_PROG_OK) ? vst[0] : 0.0f;
        a.shift[p] = isfinite(k0) ? k0 : 0.0f;
    }
    if (status != GP_PROG_OK) {
        out[0] = make_uint2(make_ins(OP_END, 0, 0), 0u);
        a.meta[p] = ProgMeta{1, status, 0, 0, 0};
        atomicOr(a.dev_status, GP_DEV_BAD_PROGRAM);
        return;
    }

    // pass 2: drop the inside of every maximal constant-only subtree (its
    // root is met first in prefix order), then fold terminal children of
    // binary nodes (prefer the right one); a constant-only function node
    // now counts as a terminal
    for (int j = 0; j < len; ++j) {
        if (mode[j] == 3 || !kon[j] || op_arity(prog[j].op) == 0) continue;
        for (int i = j + 1; i < j + size[j]; ++i) mode[i] = 3;
    }
    for (int j = 0; j < len; ++j) {
        const int op = prog[j].op;
        if (op_arity(op) != 2 || kon[j]) continue;  // kon: dropped, or a constant now
        if (op > GP_DIV) continue;  // max and min take both operands from the stack
        const int lc = j + 1, rc = j + 1 + size[j + 1];
        if (op_arity(prog[rc].op) == 0 || kon[rc]) {
            mode[rc] = 1;
            mode[j] = 1;
        } else if (op_arity(prog[lc].op) == 0 || kon[lc]) {
            mode[lc] = 1;
            mode[j] = 2;
        }
    }

    // gradient form: the number of constants before each node in prefix
    // order; the constants under node j are [cpre[j], cpre[j + size[j]])
    uint8_t cpre[GP_MAX_LEN + 1];
    if (a.grad) {
        int k = 0;
        for (int j = 0; j < len; ++j) {
            cpre[j] = (uint8_t)min(k, GP_MAX_CONSTS);
            k += prog[j].op == GP_CONST;
        }
        cpre[len] = (uint8_t)min(k, GP_MAX_CONSTS);
    }
    // pass 3: emit in reverse-scan order
    int n = 0, depth = 0;
    bool ext = false;  // an extended-set instruction was emitted
    // gradient form: a marker word before the next word when one of its
    // operands holds constants (j_top: the node whose value is the top
    // operand, j_other: the other operand's node; -1 where the partial
    // derivative is 1 and leaves the tangents as they are)
    auto mark = [&](int j_top, int j_other, bool fresh) {
        if (!a.grad) return;
        const uint32_t tlo = j_top >= 0 ? cpre[j_top] : 0u;
        const uint32_t thi = j_top >= 0 ? cpre[j_top + size[j_top]] : 0u;
        const uint32_t olo = j_other >= 0 ? cpre[j_other] : 0u;
        const uint32_t ohi = j_other >= 0 ? cpre[j_other + size[j_other]] : 0u;
        if (tlo == thi && olo == ohi) return;
        // the two common shapes get tails of their own in the fast loop
        const uint32_t shape = (thi == tlo + 1 && olo == ohi) ? 1u
                             : (tlo == thi && ohi == olo + 1 && fresh) ? 2u : 0u;
        out[n++] = make_uint2(kGradMark | (shape << 8),
                              tlo | (thi << 5) | (olo << 10) | (ohi << 15) | ((fresh ? 1u : 0u) << 20));
    };
    sp = 0;
    for (int j = len - 1; j >= 0; --j) {
        if (mode[j] == 3) continue;  // inside a folded constant subtree
        gp_node nd = prog[j];
        if (kon[j]) {  // a constant, or the root of a constant-only subtree
            nd.op = GP_CONST;
            nd.feat = 0;
            nd.c = kval[j];
        }
        const int ar = op_arity(nd.op);
        if (ar == 0) {
            if (mode[j]) continue;  // folded into its parent
            const bool x = nd.op == GP_VAR;
            const bool spill = sp > 0;  // the old top goes to slot sp-1
            const uint32_t op = (spill ? (x ? OP_PUSH_X_SP : OP_PUSH_C_SP) : (x ? OP_PUSH_X : OP_PUSH_C)) |
                                ((x && nd.feat == 1) ? kOpCol1 : 0u);
            if (!x) mark(-1, j, true);  // the constant's own tangent starts at 1
            const uint32_t w = make_ins(op, spill ? sp - 1 : 0, x ? (uint32_t)(uint16_t)nd.feat : 0u);
            out[n++] = make_uint2(w, __float_as_uint(nd.c));
            ++sp;
        } else if (ar == 1) {
            const bool e = nd.op > GP_INV;  // extended function: its number in the feature field
            ext |= e;
            mark(j + 1, -1, false);
            out[n++] = make_uint2(e ? make_ins(OP_EXT1, 0, (uint32_t)(nd.op - GP_SQ))
                                    : make_ins(OP_SQRT + (nd.op - GP_SQRT), 0, 0),
                                  0u);
        } else {
            // add, sub, mul, div, max, min
            const int b = nd.op <= GP_DIV ? nd.op - GP_ADD : 4 + (nd.op - GP_MAX);
            const int lc = j + 1, rc = j + 1 + size[j + 1];
            if (mode[j] == 0) {
                // right operand in slot sp-2, left operand is t (add: both
                // partials 1; sub: 1 for t)
                const uint32_t ops[6] = {OP_ADD_S, OP_SUB_S, OP_MUL_S, OP_DIV_S, OP_EXT2, OP_EXT2};
                ext |= b >= 4;
                if (b != 0) mark(b == 1 ? -1 : lc, rc, false);
                out[n++] = make_uint2(make_ins(ops[b], sp - 2, b >= 4 ? (uint32_t)(b - 4) : 0u), 0u);
                --sp;
            } else {
                const int tj = (mode[j] == 1) ? rc : lc;  // the inline terminal
                gp_node t = prog[tj];
                if (kon[tj]) {
                    t.op = GP_CONST;
                    t.feat = 0;
                    t.c = kval[tj];
                }
                const int x = (t.op == GP_VAR) ? 0 : 1;  // X or C variant
                // right terminal: t = op(t, u); left terminal: t = op(u, t)
                // (add, and sub with the terminal on the right, leave the
                // top's tangents as they are)
                const uint32_t fwd[4] = {OP_ADD_X, OP_SUB_X, OP_MUL_X, OP_DIV_X};
                const uint32_t rev[4] = {OP_ADD_X, OP_RSUB_X, OP_MUL_X, OP_RDIV_X};
                const int jt = (mode[j] == 1) ? lc : rc;  // the top operand's node
                mark((b == 0 || (b == 1 && mode[j] == 1)) ? -1 : jt, tj, x == 1);
                const uint32_t op = (((mode[j] == 1) ? fwd[b] : rev[b]) + x) |
                                    ((x == 0 && t.feat == 1) ? kOpCol1 : 0u);
                const uint32_t w = make_ins(op, 0, x == 0 ? (uint32_t)(uint16_t)t.feat : 0u);
                out[n++] = make_uint2(w, __float_as_uint(t.c));
            }
        }
        if (sp > depth) depth = sp;
    }
    out[n++] = make_uint2(make_ins(OP_END, 0, 0), 0u);
    a.meta[p] = ProgMeta{n, GP_PROG_OK, (int16_t)depth, (int16_t)(ext ? 1 : 0), n_consts};
}

cudaError_t launch_compile(const CompileArgs &a, cudaStream_t st) {
    if (a.n_progs <= 0) return cudaSuccess;
    const int block = 128;
    const int grid = (a.n_progs + block - 1) / block;
    compile_kernel<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

// Counting sort of program ids: key = class * 256 + (256 - n_ins), so the
// classes follow one another (0, 1, 2, 3) and, inside a class, longer programs
// come first (longest-processing-time order for the dynamic work queue).
// mode 0: the evaluator's classes (stack depth, extended functions); mode
// 1: the gradient's buckets (constants, stack depth), whose programs with
// their marker words may exceed 256 words (those share the first key).
// Invalid programs (n_ins = 1) land at the end of class 0.  Order inside
// one key is arbitrary; results do not depend on it.
constexpr int kOrderBins = kOrderClasses * 256;

__device__ __forceinline__ int order_class(const ProgMeta &m, int mode) {
    return mode == 0 ? prog_class(m.depth, m.ext) : grad_bucket(m.n_consts, m.depth, m.ext);
}

__global__ void __launch_bounds__(1024) order_kernel(const ProgMeta *meta, int n_progs,
                                                     int32_t *order, int32_t *class_count,
                                                     int mode, int edge) {
    __shared__ int hist[kOrderBins];
    __shared__ int cursor[kOrderBins];
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < n_progs; p += blockDim.x) {
        const ProgMeta m = meta[p];
        const int cls = order_class(m, mode);
        const int key = cls * 256 + (256 - min(m.n_ins, 256));
        atomicAdd(&hist[key], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0, prev = 0;
        for (int i = 0; i < kOrderBins; ++i) {
            cursor[i] = run;
            run += hist[i];
            if (i % 256 == 255) {
                class_count[i / 256] = run - prev;
                prev = run;
            }
        }
        // class-0 programs longer than edge: keys 0 .. 255 - edge (n_ins > edge)
        int n_long = 0;
        if (edge > 0)
            for (int k = 0; k < 256 - edge; ++k) n_long += hist[k];
        class_count[kOrderClasses] = n_long;
        class_count[kOrderClasses + 1] = 0;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n_progs; p += blockDim.x) {
        const ProgMeta m = meta[p];
        const int cls = order_class(m, mode);
        const int key = cls * 256 + (256 - min(m.n_ins, 256));
        const int pos = atomicAdd(&cursor[key], 1);
        order[pos] = p;
    }
}

cudaError_t launch_order(const ProgMeta *meta, int n_progs, int32_t *order,
                         int32_t *class_count, cudaStream_t st, int mode, int edge) {
    order_kernel<<<1, 1024, 0, st>>>(meta, n_progs, order, class_count, mode, edge);
    return cudaGetLastError();
}

// Total weight in FP64 with a fixed partition: block b sums rows
// [b*span, (b+1)*span) with a fixed per-thread stride and a fixed tree, and
// one warp then adds the block sums in order.  w == NULL gives n_rows.
__global__ void __launch_bounds__(256) sumw_kernel(const float *__restrict__ w, int64_t n_rows,
                                                   double *part) {
    __shared__ double red[256];
    const int64_t span = (n_rows + kSumwBlocks - 1) / kSumwBlocks;
    const int64_t r0 = (int64_t)blockIdx.x * span;
    const int64_t r1 = min(n_rows, r0 + span);
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += (double)w[r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sumw_final_kernel(const double *part, double *sumw, const float *w,
                                  int64_t n_rows) {
    if (threadIdx.x != 0) return;
    if (w == nullptr) {
        *sumw = (double)n_rows;
        return;
    }
    double s = 0.0;
    for (int i = 0; i < kSumwBlocks; ++i) s += part[i];
    *sumw = s;
}

cudaError_t launch_sumw(const float *w, int64_t n_rows, double *part, double *sumw,
                        cudaStream_t st) {
    if (w) sumw_kernel<<<kSumwBlocks, 256, 0, st>>>(w, n_rows, part);
    sumw_final_kernel<<<1, 32, 0, st>>>(part, sumw, w, n_rows);
    return cudaGetLastError();
}

// Statistics of y for the correlation fitness, with the partition of
// sumw_kernel: phase 0 sums w y per block; the first final step sets
// ybar = sum w y / sum w (FP64) and its float rounding; phase 1 sums
// w yc and w yc^2 per block with yc = fl(y - fl(ybar)), the very values the
// evaluator forms; the second final step adds the block sums in order.
template <int PHASE>
__global__ void __launch_bounds__(256) ystats_kernel(const float *__restrict__ y,
                                                     const float *__restrict__ w, int64_t n_rows,
                                                     const double *ystat, double *part) {
    __shared__ double red[2][256];
    const int64_t span = (n_rows + kSumwBlocks - 1) / kSumwBlocks;
    const int64_t r0 = (int64_t)blockIdx.x * span;
    const int64_t r1 = min(n_rows, r0 + span);
    const float ybar = PHASE ? (float)ystat[3] : 0.0f;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const double wr = w ? (double)w[r] : 1.0;
        if (PHASE == 0) {
            s0 += wr * (double)y[r];
        } else {
            const double yc = (double)__fsub_rn(y[r], ybar);
            s0 += wr * yc;
            s1 += wr * yc * yc;
        }
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = red[0][0];
        part[2 * blockIdx.x + 1] = red[1][0];
    }
}

template <int PHASE>
__global__ void ystats_final_kernel(const double *part, const double *sumw, double *ystat) {
    if (threadIdx.x != 0) return;
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < kSumwBlocks; ++i) {
        s0 += part[2 * i];
        s1 += part[2 * i + 1];
    }
    if (PHASE == 0) {
        const double ybar = s0 / *sumw;
        ystat[0] = ybar;
        ystat[3] = (double)(float)ybar;
    } else {
        ystat[1] = s0;
        ystat[2] = s1;
    }
}

cudaError_t launch_ystats(const float *y, const float *w, int64_t n_rows, const double *sumw,
                          double *part, double *ystat, cudaStream_t st) {
    ystats_kernel<0><<<kSumwBlocks, 256, 0, st>>>(y, w, n_rows, ystat, part);
    ystats_final_kernel<0><<<1, 32, 0, st>>>(part, sumw, ystat);
    ystats_kernel<1><<<kSumwBlocks, 256, 0, st>>>(y, w, n_rows, ystat, part);
    ystats_final_kernel<1><<<1, 32, 0, st>>>(part, sumw, ystat);
    return cudaGetLastError();
}

}  // namespace gpk
