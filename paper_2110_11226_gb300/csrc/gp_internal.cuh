// gp_internal.cuh -- definitions shared by the translation units of libgp.
//
// Compiled program form.  The device pre-pass turns each prefix list into a
// sequence of register-stack instructions, in reverse-scan order (Sec.
// III-A: the list is evaluated by scanning it from the end).  The top of
// the stack lives in a register array `t`; deeper values in a register
// array `s[slot]`.  Each instruction names its slot at compile time so the
// interpreter can address registers with constant indices:
//   PUSH_X(k)/PUSH_C(k)  stack height k before the push: s[k-1] = t (k>0),
//                        t = X[feat] / c
//   BIN(op, k)           t = op(t, s[k])      (left = t, first pop)
//   UN(op)               t = op(t)
//   BIN_RX/RC(op)        t = op(t, X[feat] / c)  right child is a terminal
//   BIN_LX/LC(op)        t = op(X[feat] / c, t)  left child is a terminal
//   END
// The folded forms evaluate the same operations on the same operands as
// the plain reverse scan, so every result is bit-identical to it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gp.h"

namespace gpk {

constexpr int kCodeStride = 256;   // instructions per program (255 + END)
constexpr int kEvalBlockThreads = 256;  // threads per block of the evaluator
constexpr uint32_t kNeedsX = 0x100u;  // instruction bit 8: reads X[feat]
constexpr int kDeepSlots = GP_MAX_STACK - 1;  // s[0..18]
constexpr float kThr = 0.001f;     // protected-operator threshold

// instruction ids (low 8 bits of ins.x; feature index in the high 16 bits)
enum : uint32_t {
    K_PUSH_X = 0,                     // + k, k = 0..19
    K_PUSH_C = 20,                    // + k
    K_BIN = 40,                       // + b*19 + k, b = op - GP_ADD (0..3)
    K_UN = K_BIN + 4 * kDeepSlots,    // 116 + (op - GP_SQRT), 9 unary ops
    K_BIN_RX = K_UN + 9,              // 125 + b
    K_BIN_RC = K_BIN_RX + 4,          // 129 + b
    K_BIN_LX = K_BIN_RC + 4,          // 133 + b
    K_BIN_LC = K_BIN_LX + 4,          // 137 + b
    K_END = K_BIN_LC + 4,             // 141
    K_COUNT = K_END + 1
};

// per-program metadata written by the pre-pass
struct ProgMeta {
    int32_t n_ins;     // instructions including END
    int32_t status;    // gp_prog_status
    int32_t depth;     // largest stack height of the compiled form
    int32_t n_consts;  // CONST nodes
};

// depth classes: programs whose compiled stack fits kSmallDepth run in a
// kernel instance with fewer deep register slots
constexpr int kSmallDepth = 8;     // s[0..6] + t
constexpr int kNumClasses = 2;

// Workspace carved out of one device allocation (all offsets 256-aligned).
struct Workspace {
    unsigned long long *counters;  // [8] work-queue counters
    double *sumw;                  // [1] total weight
    double *sumw_part;             // [kSumwBlocks]
    uint2 *code;                   // [P][kCodeStride]
    ProgMeta *meta;                // [P]
    int32_t *order;                // [P] program ids, by class then length
    int32_t *class_count;          // [kNumClasses + 2]
    float *part;                   // [P][n_chunks] per-item partial sums
    // constant-gradient extras (may be null)
    uint8_t *rchild;               // [P][256] right child offset per node
    int8_t *kslot;                 // [P][256] constant slot per node or -1
    int16_t *cnode;                // [P][16] node index of constant k
    float *gpart;                  // [P][n_chunks][16]
    size_t bytes;
};

constexpr int kSumwBlocks = 512;

struct Layout {
    size_t counters, sumw, sumw_part, code, meta, order, class_count, part;
    size_t rchild, kslot, cnode, gpart, total;
};

Layout make_layout(int n_progs, int n_chunks, bool grad);
Workspace carve(void *base, const Layout &L, bool grad);

// ---- kernels / launchers (defined in the .cu files) --------------------
struct CompileArgs {
    const gp_node *progs;
    const int32_t *offsets;
    int n_progs;
    int n_feat;
    uint2 *code;
    ProgMeta *meta;
    uint8_t *rchild;   // optional
    int8_t *kslot;     // optional
    int16_t *cnode;    // optional
    unsigned int *dev_status;
    int32_t *out_prog_status;  // optional, caller's
};
cudaError_t launch_compile(const CompileArgs &a, cudaStream_t st);
cudaError_t launch_order(const ProgMeta *meta, int n_progs, int32_t *order,
                         int32_t *class_count, cudaStream_t st);
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
    unsigned long long *counter;
    float *part;       // eval mode
    float *pred;       // predict mode
    unsigned int *dev_status;
    int vec_ok;
};
// One launcher per (rows per thread, feature mode) instance; a.cls picks
// the depth class (register slots).  fmode 2: columns 0 and 1 held in
// registers (n_feat <= 2); fmode 0: feature columns loaded per reference.
// info_*: resident blocks per SM for `block` threads; *regs = registers.
#define GP_EVAL_INSTANCE(R, F)                                                  \
    cudaError_t launch_eval_r##R##_f##F(const EvalArgs &a, int grid, int block, \
                                        cudaStream_t st);                       \
    int info_eval_r##R##_f##F(int cls, int block, int *regs);
GP_EVAL_INSTANCE(4, 2)
GP_EVAL_INSTANCE(4, 0)
GP_EVAL_INSTANCE(8, 2)
GP_EVAL_INSTANCE(8, 0)
#undef GP_EVAL_INSTANCE
cudaError_t launch_predict(const EvalArgs &a, int grid, int block,
                           cudaStream_t st);
int info_predict(int block, int *regs);

struct FinalizeArgs {
    const float *part;
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
    const gp_node *progs;
    const int32_t *offsets;
    const ProgMeta *meta;
    const int32_t *order;
    const uint8_t *rchild;
    const int8_t *kslot;
    const float *X;
    int64_t ld;
    int64_t n_rows;
    const float *y;
    const float *w;
    int n_progs;
    int metric;
    int64_t chunk_rows;
    int n_chunks;
    unsigned long long *counter;
    float *part;   // [P][n_chunks] loss sums
    float *gpart;  // [P][n_chunks][16]
    unsigned int *dev_status;
};
cudaError_t launch_grad(const GradArgs &a, int grid, int block,
                        cudaStream_t st);
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
    const int16_t *cnode;
    int n_progs;
    const float *grad;
    float *m;
    float *v;
    int step;
    float lr, beta1, beta2, eps;
};
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st);

cudaError_t probe_pipes(double *out, cudaStream_t st);

}  // namespace gpk
