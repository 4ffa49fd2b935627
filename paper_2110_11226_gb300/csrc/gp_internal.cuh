// gp_internal.cuh -- definitions shared by the translation units of libgp.
//
// Compiled program form.  The device pre-pass turns each prefix list into a
// sequence of stack-machine instructions in reverse-scan order (Sec. III-A:
// the list is evaluated by scanning it from the end).  The top of the stack
// lives in registers (t); deeper values live in a per-warp shared-memory
// stack whose slot numbers the pre-pass resolves.  Each instruction is one
// of 30 operations that name their operand source, or one of two entries
// for the extended functions, so the interpreter's only branch per
// instruction is one switch:
//   PUSH_X / PUSH_C        t = X[feat] / c
//   PUSH_X_SP / PUSH_C_SP  stack[slot] = t first (push onto a non-empty stack)
//   op_S                   t = op(t, stack[slot])      (right operand popped)
//   op_X / op_C            t = op(t, X[feat] / c)      (right child a terminal)
//   RSUB_*, RDIV_*         t = op(X[feat] / c, t)      (left child a terminal)
//   unary                  t = f(t)
//   END
// A binary node whose right child is a terminal takes it inline; failing
// that, one whose left child is a terminal takes it inline with the
// reversed operation (add and mul commute exactly in IEEE arithmetic);
// otherwise its right operand sits in a stack slot, as it always does for
// max and min.  These forms evaluate
// the same operations on the same operands as the plain reverse scan, so
// every result is bit-identical to it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp.h"

namespace gpk {

constexpr int kCodeStride = 256;   // instructions per program (255 + END)
constexpr int kEvalBlockThreads = 256;  // threads per block of the evaluator
constexpr int kDeepSlots = GP_MAX_STACK - 1;  // s[0..18]
constexpr float kThr = 0.001f;     // protected-operator threshold

// instruction word x: op in bits 0-4; bit 5 set on a column read of
// column 1 (the fast loop's dispatch index is bits 0-5, so with the two
// columns held in registers each column has its own table entry); stack
// slot in bits 8-15; feature index (column reads) or extended function
// number (EXT1, EXT2) in bits 16-31.  Word y: the constant.
enum : uint32_t {
    OP_PUSH_X = 0, OP_PUSH_C = 1, OP_PUSH_X_SP = 2, OP_PUSH_C_SP = 3,
    OP_ADD_S = 4, OP_SUB_S = 5, OP_MUL_S = 6, OP_DIV_S = 7,
    OP_ADD_X = 8, OP_ADD_C = 9, OP_SUB_X = 10, OP_SUB_C = 11,
    OP_RSUB_X = 12, OP_RSUB_C = 13, OP_MUL_X = 14, OP_MUL_C = 15,
    OP_DIV_X = 16, OP_DIV_C = 17, OP_RDIV_X = 18, OP_RDIV_C = 19,
    OP_SQRT = 20, OP_LOG = 21, OP_EXP = 22, OP_SIN = 23, OP_COS = 24,
    OP_TAN = 25, OP_ABS = 26, OP_NEG = 27, OP_INV = 28, OP_END = 29,
    // the extended function set behind two entries, the function in bits
    // 16-18: EXT1 unary (sq, cube, cbrt, tanh, atan, sinh, cosh), EXT2
    // binary (max, min; the right operand always in a stack slot)
    OP_EXT1 = 30, OP_EXT2 = 31
};
constexpr uint32_t kOpCol1 = 32;  // bit 5: a column read of column 1

// Gradient form of a program (forward-mode derivatives with respect to its
// constants).  The constants are numbered 0, 1, ... in prefix order, so the
// constants under any node form a contiguous range of numbers, and those
// of a binary node's left subtree come just before those of its right one.
// The tangent of constant k on a row, dt[k], is the derivative with
// respect to c_k of the stack value whose subtree holds c_k; a word that
// combines its operands multiplies the tangents under each operand by the
// word's partial derivative with respect to that operand, so at the end
// dt[k] is d(program)/d(c_k).  Each word whose operands hold constants is
// preceded by a marker word: x = kGradMark | shape << 8 (shape 1: one
// constant under t and none under the other operand; 2: none under t and
// one fresh constant; 0: anything else), y = the ranges
//   bits 0-4 / 5-9    [tlo, thi): constants under the top operand t
//   bits 10-14 / 15-19 [olo, ohi): constants under the other operand (the
//                      popped slot, the inline terminal, or for a push of a
//                      constant the constant itself)
//   bit 20            fresh: the other operand is a constant terminal, its
//                      tangent starts at 1 here
// The marker's low five bits read as OP_END, and the fast loop hands it
// back like any word it does not run.
constexpr uint32_t kGradMark = OP_END | kOpCol1;
constexpr int kGradCodeStride = 512;  // words of the gradient form (<= 2 per node + END)
enum : uint32_t { EXT_SQ = 0, EXT_CUBE, EXT_CBRT, EXT_TANH, EXT_ATAN, EXT_SINH, EXT_COSH };
enum : uint32_t { EXT_MAX = 0, EXT_MIN = 1 };

__host__ __device__ constexpr uint32_t make_ins(uint32_t op, uint32_t slot, uint32_t feat) {
    return op | (slot << 8) | (feat << 16);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key advanced by the Weyl constants between rounds.
static __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// per-program metadata written by the pre-pass
struct ProgMeta {
    int32_t n_ins;     // instructions including END
    int32_t status;    // gp_prog_status
    int16_t depth;     // largest stack height of the compiled form
    int16_t ext;       // 1: uses an extended function (EXT1/EXT2 words)
    int32_t n_consts;  // CONST nodes
};

// Program classes, one evaluator instance each.  Programs without the
// extended functions whose compiled stack fits kShallowDepth form class 0,
// the common one: a 6-slot shared-memory stack, so that at 8 rows per
// thread 4 blocks of 8 warps fit per SM (a 7-slot stack fits 3).  Those of
// depth kSmallDepth form class 3 (7 slots, 4 rows per thread); programs
// with the extended functions and a stack of at most kSmallDepth, class 2
// (7 slots; their dispatch entries would slow class 0 down); deeper
// programs, class 1 (19 slots, every function).
constexpr int kSmallDepth = 8;     // 7 stack slots + t
constexpr int kShallowDepth = 7;   // 6 stack slots + t
constexpr int kNumClasses = 4;
constexpr int kClassShallow = 0, kClassDeep = 1, kClassShallowExt = 2, kClassShallow8 = 3;
__host__ __device__ inline int prog_class(int depth, int ext) {
    if (depth > kSmallDepth) return kClassDeep;
    if (ext) return kClassShallowExt;
    return depth > kShallowDepth ? kClassShallow8 : kClassShallow;
}

// Buckets of the constant gradient, one launch each: the tangents of a
// warp's rows take kGradTan0 (bucket 0), kGradTan1 (bucket 1) or
// GP_MAX_CONSTS (buckets 2, 3) shared-memory slots per row, the value
// stack 7 (buckets 0-2) or 19 (bucket 3); fewer tangent slots leave room
// for more resident warps.
// Programs without constants (and without the extended functions, stack
// depth <= 8) need no tangents: they form order class kGradBuckets and
// run through the evaluator, which writes their loss partials.
constexpr int kGradBuckets = 4;
constexpr int kGradTan0 = 4, kGradTan1 = 8;
__host__ __device__ inline int grad_bucket(int n_consts, int depth, int ext) {
    if (depth > kSmallDepth) return 3;
    if (n_consts == 0 && !ext) return kGradBuckets;
    return n_consts <= kGradTan0 ? 0 : (n_consts <= kGradTan1 ? 1 : 2);
}
// classes of the program order (evaluator classes or gradient buckets)
constexpr int kOrderClasses = 5;

// Workspace carved out of one device allocation (all offsets 256-aligned).
struct Workspace {
    unsigned long long *counters;  // [8] work-queue counters
    double *sumw;                  // [1] total weight
    double *sumw_part;             // [kSumwBlocks]
    uint2 *code;                   // [P][kCodeStride], the gradient form [P][kGradCodeStride]
    ProgMeta *meta;                // [P]
    int32_t *order;                // [P] program ids, by class then length
    int32_t *class_count;          // [kOrderClasses + 2]
    float *part;                   // [P][n_chunks] per-item partial sums
    // correlation extras (may be null)
    double *ystat;                 // [4]: ybar, sum w yc, sum w yc^2, (float) ybar
    double *ystat_part;            // [kSumwBlocks][2]
    float *shift;                  // [P] program value at row 0
    double *mom;                   // [P][n_chunks][3] per-item moment sums
    // constant-gradient extra (may be null)
    float *gpart;                  // [P][n_chunks][16]
    size_t bytes;
};

constexpr int kSumwBlocks = 512;

struct Layout {
    size_t counters, sumw, sumw_part, code, meta, order, class_count, part;
    size_t ystat, ystat_part, shift, mom;
    size_t gpart, total;
};

// moments: reserve the correlation extras (GP_PEARSON)
Layout make_layout(int n_progs, int n_chunks, bool grad, bool moments = false);
Workspace carve(void *base, const Layout &L, bool grad);

// forget the cached device addresses of gp_evaluate_static's array
void static_scratch_forget();

// workspace bytes of one batched evaluation with this metric (0 for bad
// arguments); gp_workspace_size reports the largest over all metrics
size_t workspace_bytes_for(int n_progs, int64_t n_rows, int n_feat, const gp_eval_opts *opts,
                           int metric);

// ---- kernels / launchers (defined in the .cu files) --------------------
struct CompileArgs {
    const gp_node *progs;
    const int32_t *offsets;
    int n_progs;
    int n_feat;
    uint2 *code;
    ProgMeta *meta;
    unsigned int *dev_status;
    int32_t *out_prog_status;  // optional, caller's
    // optional: each program's value at row 0 of X (column stride ld)
    const float *X;
    int64_t ld;
    float *shift;
    // gradient form (code stride kGradCodeStride): no constant-only subtree
    // is folded, so every constant keeps a word of its own or an operand
    // place, and a marker word (kGradMark) precedes each word whose
    // operands carry constants (see kGradMark)
    int grad;
};
cudaError_t launch_compile(const CompileArgs &a, cudaStream_t st);
// weighted mean of y and the moments of yc = fl(y - fl(ybar)) (FP64,
// fixed partition); needs the total weight already in *sumw
cudaError_t launch_ystats(const float *y, const float *w, int64_t n_rows, const double *sumw,
                          double *part, double *ystat, cudaStream_t st);
// mode 0 with edge > 0 also writes to class_count[kOrderClasses] how many
// class-0 programs have more than `edge` compiled words (the long bucket,
// which the order puts first)
cudaError_t launch_order(const ProgMeta *meta, int n_progs, int32_t *order,
                         int32_t *class_count, cudaStream_t st, int mode = 0, int edge = 0);
cudaError_t launch_sumw(const float *w, int64_t n_rows, double *part,
                        double *sumw, cudaStream_t st);

struct EvalArgs {
    const uint2 *code;
    const ProgMeta *meta;
    const int32_t *order;
    const int32_t *class_count;
    int cls;
    const float *X;
    int64_t ld;
    int64_t n_rows;
    const float *y;
    const float *w;
    int n_progs;
    int metric;
    int64_t chunk_rows;
    int n_chunks;
    // 0: the whole class; 1, 2: the long, the short programs of class 0
    // (class_count[kOrderClasses] long ones first)
    int sub;
    unsigned long long *counter;
    float *part;       // eval mode
    float *pred;       // predict mode
    unsigned int *dev_status;
    int vec_ok;
    // moments mode (correlation fitness): per-item sums of w d, w d^2 and
    // w d yc with d = p - shift[p], yc = y - ybar
    double *mom;
    const float *shift;
    const double *ystat;
    // 0: programs' words every kCodeStride entries; else this stride
    int code_stride;
    // 0: the programs of class cls; k + 1: those of order class k (the
    // constant gradient's buckets: its constant-free programs)
    int qcls;
};
// One launcher per (rows per thread, feature mode) instance; a.cls picks
// the program class (stack slots, extended functions).  fmode 2: columns 0 and 1 held in
// registers (n_feat <= 2); fmode 0: feature columns loaded per reference.
// info_*: resident blocks per SM for `block` threads; *regs = registers.
#define GP_EVAL_INSTANCE(R, F)                                                  \
    cudaError_t launch_eval_r##R##_f##F(const EvalArgs &a, int grid, int block, \
                                        cudaStream_t st);                       \
    int info_eval_r##R##_f##F(int cls, int block, int *regs, bool moments);
GP_EVAL_INSTANCE(4, 2)
GP_EVAL_INSTANCE(4, 0)
GP_EVAL_INSTANCE(16, 2)
GP_EVAL_INSTANCE(16, 0)
#undef GP_EVAL_INSTANCE
// 8 rows per thread: class 0 only, with the store epilogue too (pred)
cudaError_t launch_eval_r8_f2(const EvalArgs &a, int grid, int block, cudaStream_t st);
int info_eval_r8_f2(int cls, int block, int *regs, bool moments, bool pred = false);
cudaError_t launch_eval_r8_f0(const EvalArgs &a, int grid, int block, cudaStream_t st);
int info_eval_r8_f0(int cls, int block, int *regs, bool moments, bool pred = false);
cudaError_t launch_predict(const EvalArgs &a, int grid, int block,
                           cudaStream_t st);
int info_predict(int cls, int block, int *regs);
// the same for tables of at most two columns (feature mode 2)
cudaError_t launch_predict_f2(const EvalArgs &a, int grid, int block, cudaStream_t st);
int info_predict_f2(int cls, int block, int *regs);

struct FinalizeArgs {
    const float *part;
    const double *mom;     // moments mode (GP_PEARSON) instead of part
    const double *ystat;
    int n_chunks;
    int n_progs;
    const ProgMeta *meta;
    const double *sumw;
    int metric;
    int accum;
    float *out;
    double *out64;
    int32_t *out_prog_status;
};
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t st);

struct PlainArgs {
    const gp_node *progs;
    const int32_t *offsets;
    const ProgMeta *meta;
    const float *X;
    int64_t ld;
    int64_t n_rows;
    const float *y;
    const float *w;
    int metric;
    int n_blocks;   // row blocks of 256
    float *part;    // [P][n_blocks]
};
cudaError_t launch_plain(const PlainArgs &a, int p, cudaStream_t st);

struct TournArgs {
    const float *fitness;
    const int32_t *offsets;
    int n_progs;
    int n_tourn;
    int k;
    float parsimony;
    int greater;
    uint64_t seed;
    uint64_t offset;
    int32_t *out;
};
cudaError_t launch_tournament(const TournArgs &a, cudaStream_t st);

struct GradArgs {
    const uint2 *code;          // gradient form (CompileArgs::grad), [P][kGradCodeStride]
    const ProgMeta *meta;
    const int32_t *order;       // by bucket, then length
    const int32_t *class_count; // programs per bucket
    int bucket;                 // the launch's bucket (grad_bucket)
    const float *X;
    int64_t ld;
    int64_t n_rows;
    int n_feat;
    const float *y;
    const float *w;
    int metric;
    int64_t chunk_rows;
    int n_chunks;
    unsigned long long *counter;  // [kGradBuckets] work-queue counters, one per bucket
    int vec_ok;                   // X, y, w and the row counts allow 16-byte row loads
    float *part;   // [P][n_chunks] loss sums
    float *gpart;  // [P][n_chunks][16]
    unsigned int *dev_status;
};
// one launch of bucket a.bucket filling every SM; with occ non-null only
// reports the resident blocks per SM (no launch)
cudaError_t launch_grad(const GradArgs &a, int sms, cudaStream_t st, int *occ = nullptr);
struct GradFinalizeArgs {
    const float *part;
    const float *gpart;
    int n_chunks;
    int n_progs;
    const ProgMeta *meta;
    const double *sumw;
    int metric;
    float *grad;
    float *fit;
};
cudaError_t launch_grad_finalize(const GradFinalizeArgs &a, cudaStream_t st);

struct AdamArgs {
    gp_node *progs;
    const int32_t *offsets;
    const ProgMeta *meta;
    int n_progs;
    const float *grad;
    float *m;
    float *v;
    int step;
    float lr, beta1, beta2, eps;
};
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st);

// constants <-> a dense [n_progs][GP_MAX_CONSTS] array (prefix order);
// to_nodes = false gathers (missing slots 0), true scatters
cudaError_t launch_consts(gp_node *progs, const int32_t *offsets, int n_progs, float *consts,
                          bool to_nodes, cudaStream_t st);

cudaError_t probe_pipes(double *out, cudaStream_t st);
// Spearman fitness (gp_rank.cu): scratch bytes for n_seg segments of n
// values; the target's doubled ranks by row and its per-tile weighted rank
// sums (target_part_bytes(n) bytes); one batch of predictions [n_seg][n]
// to fitness
size_t rank_scratch_bytes(int n_seg, int64_t n);
size_t target_part_bytes(int64_t n);
cudaError_t target_ranks(const float *y, const float *w, int64_t n, void *scratch, uint32_t *r2y,
                         double *tpart, cudaStream_t st);
cudaError_t spearman_batch(const float *pred, int n_seg, int64_t n, const uint32_t *r2y,
                           const double *tpart, const float *w, void *scratch, float *out,
                           double *out64, cudaStream_t st);

// device-side mutation (gp_mutate)
struct MutArgs {
    const gp_node *progs;
    const int32_t *offsets;
    int n_progs;
    int n_feat;
    const int32_t *parents;  // [2 n_out]
    int n_out;
    uint64_t thr[4];         // cumulative kind thresholds, floor(p 2^32)
    uint64_t thr_replace;    // point mutation, per node
    int subtree_depth;
    int n_funcs, n_unary, n_binary;
    int16_t funcs[GP_NUM_OPS], unary[GP_NUM_OPS], binary[GP_NUM_OPS];  // allowed, by arity
    uint64_t seed, offset;
    gp_node *scratch;        // [n_out][256] children
    int32_t *lens;           // [n_out]
    int32_t *kind;           // [n_out] or null
    gp_node *out;
    int32_t *out_offsets;    // [n_out + 1]
    unsigned int *dev_status;
};
cudaError_t launch_mutate(const MutArgs &a, cudaStream_t st);


}  // namespace gpk
