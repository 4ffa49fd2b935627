/*
 * gp.h -- C ABI of libgp: batched fitness evaluation and selection for
 * stack-based genetic programming on one GB300 GPU (sm_103a).
 *
 * The method is that of Sathia, Ganesh and Nanditale, "Accelerating Genetic
 * Programming using GPUs" (arXiv 2110.11226):
 *   - a program is a prefix (Polish) list of nodes evaluated with a stack
 *     by scanning the list in reverse (Sec. III-A);
 *   - every program is evaluated on every row of a column-major dataset
 *     that already resides in GPU memory (Sec. III, III-C3);
 *   - a weighted loss per row is reduced to one raw fitness per program
 *     (Sec. III-C3);
 *   - tournament selection draws k programs per tournament with Philox and
 *     keeps the best adjusted fitness, adjusted = raw + c * len
 *     (Sec. III-C1, Eqs. parsimony and fitness).
 * The constant-gradient and Adam entry points have no counterpart in the
 * paper; they tune the ephemeral constants of the programs.
 *
 * Conventions for every entry point:
 *   - Pointers are device pointers unless the comment says "host"; they are
 *     owned by the caller and never freed or retained by the library.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; nothing synchronises
 *     unless the comment says so.
 *   - The return value is GP_OK (0) or a negative gp_status.  Argument
 *     errors are returned before anything is launched.  Problems found on
 *     the device (a malformed program) never trap: they set bits of a
 *     device status word (gp_last_device_status) and NaN results.
 *   - Floating point: evaluation in FP32 (IEEE +,-,*,/ and sqrt, CUDA's
 *     accurate libm functions, no contraction into FMA); the cross-block
 *     fitness sum in FP64.
 */
#ifndef GP_H_
#define GP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GP_MAX_STACK 20   /* stack slots: a program must never hold more    */
#define GP_MAX_LEN 255    /* nodes per program                              */
#define GP_MAX_CONSTS 16  /* constants per program for gp_const_grad        */

/* One node of a prefix list (8 bytes).  VAR reads column `feat` of X;
 * CONST pushes `c`; functions ignore feat and c. */
typedef struct gp_node {
    int16_t op;
    int16_t feat;
    float c;
} gp_node;

/* Function set: arity <= 2 (Sec. III).  Binary functions take the first
 * value popped in the reverse scan as their LEFT operand, so the prefix
 * list [SUB, x0, x1] computes x0 - x1.  Protected operators use the
 * threshold 0.001f with the strict test |v| < 0.001f:
 *   DIV(a,b) = 1 on the protected branch, INV(a) = 0, LOG(a) = 0,
 *   otherwise a/b, 1/a, log|a|; SQRT(a) = sqrt|a|.
 * Beyond the paper's benchmark set {+,-,*,/,sin,cos,tan} (whose full list
 * of 33 functions the paper does not give): SQ(a) = a*a, CUBE(a) = (a*a)*a
 * (each product rounded), CBRT, TANH, ATAN, SINH, COSH (CUDA's float
 * functions, unprotected), MAX(a,b) / MIN(a,b) = the larger / smaller
 * operand, NaN if either is NaN, the right operand when they compare
 * equal.  Unary ops are 6..21, binary 2..5 and 22..23. */
enum gp_op {
    GP_CONST = 0, GP_VAR = 1,
    GP_ADD = 2, GP_SUB = 3, GP_MUL = 4, GP_DIV = 5,
    GP_SQRT = 6, GP_LOG = 7, GP_EXP = 8, GP_SIN = 9, GP_COS = 10,
    GP_TAN = 11, GP_ABS = 12, GP_NEG = 13, GP_INV = 14,
    GP_SQ = 15, GP_CUBE = 16, GP_CBRT = 17, GP_TANH = 18, GP_ATAN = 19,
    GP_SINH = 20, GP_COSH = 21, GP_MAX = 22, GP_MIN = 23,
    GP_NUM_OPS = 24
};

/* Fitness metrics (Sec. III-C3), weighted means over the rows:
 *   MAE  = sum w|p-y| / sum w          MSE = sum w (p-y)^2 / sum w
 *   RMSE = sqrt(MSE)                   LOGLOSS = sum w l(p,y) / sum w
 * with l(p,y) = c|p| + log1p(exp(-|p|)), c = 1-y if p >= 0 else y (the
 * logistic loss of sigmoid(p) against a label y in {0,1}; the c|p| term
 * is 0 when c == 0).  These four are smaller-is-better.
 *   PEARSON = |r_w(p, y)|, the absolute weighted Karl Pearson correlation
 *             cov_w(p,y) / sqrt(var_w(p) var_w(y)) with weighted means;
 *             0 when either variance is 0, NaN when a sum is not finite.
 *             Greater is better (pass greater_is_better = 1 to the
 *             tournament).  Batched evaluator only (gp_evaluate*,
 *             gp_evaluate_host, gp_evaluate_static, gp_autotune).
 *   SPEARMAN = |r_w| of the ranks: each row's prediction and target are
 *             replaced by their 1-based ranks among all rows (ties share
 *             the mean of their positions), then PEARSON of the ranks with
 *             the weights w; NaN when a prediction is NaN.  Greater is
 *             better.  gp_evaluate, gp_evaluate_ex and gp_evaluate_host
 *             only; it materialises each program's predictions and sorts
 *             them, so it is far slower than the fused metrics. */
enum gp_metric { GP_MAE = 0, GP_MSE = 1, GP_RMSE = 2, GP_LOGLOSS = 3, GP_PEARSON = 4,
                 GP_SPEARMAN = 5 };

enum gp_status {
    GP_OK = 0,
    GP_ERR_ARG = -1,       /* bad argument (NULL, size, metric, opts)     */
    GP_ERR_PROGRAM = -2,   /* malformed program (host-side validation)    */
    GP_ERR_CONSTS = -3,    /* more than GP_MAX_CONSTS constants           */
    GP_ERR_CUDA = -4,      /* a CUDA runtime call failed                  */
    GP_ERR_TIMEOUT = -5,   /* a bounded device loop hit its cap           */
    GP_ERR_NOMEM = -6,     /* device allocation failed                    */
    GP_ERR_WORKSPACE = -7  /* caller workspace too small or misaligned    */
};

/* Per-program status written by the validator (device pre-pass and
 * gp_validate_host). */
enum gp_prog_status {
    GP_PROG_OK = 0, GP_PROG_BAD_LENGTH = 1, GP_PROG_BAD_OP = 2,
    GP_PROG_BAD_FEATURE = 3, GP_PROG_UNDERFLOW = 4, GP_PROG_LEFTOVER = 5,
    GP_PROG_TOO_DEEP = 6
};

/* Bits of the device status word. */
#define GP_DEV_BAD_PROGRAM 0x1u      /* a program failed validation     */
#define GP_DEV_TOO_MANY_CONSTS 0x2u  /* gp_const_grad: > 16 constants  */
#define GP_DEV_QUEUE_CAP 0x4u        /* persistent work loop hit its cap */
#define GP_DEV_BAD_PARENT 0x8u       /* gp_mutate: parent index out of range */

/* Cross-block accumulation of the fitness sums. */
enum gp_accum { GP_ACCUM_FP64 = 0, GP_ACCUM_KAHAN32 = 1 };

/* Tunables of the batched evaluator; zero means "choose".  The choice is
 * the autotuned one for this problem shape when gp_autotune has run,
 * otherwise a fixed default.
 * Length buckets: with long_edge > 0 the programs of the common class
 * (compiled stack of at most 7 values, no extended function) whose compiled
 * form is longer than long_edge words run in a launch of their own, with
 * long_rows_per_thread and long_blocks_per_sm (0: rows_per_thread and
 * blocks_per_sm), before the shorter ones; long_edge = -1 asks for no split
 * (the default when nothing is tuned).
 * A program's fitness is bit-identical for every choice that gives it the
 * same rows per thread and the same chunk_rows (fixed reduction partition);
 * blocks_per_sm and the bucket it lands in never change it. */
typedef struct gp_eval_opts {
    int rows_per_thread;       /* 4, 8 or 16 (default 8)                      */
    int chunk_rows;            /* rows per work item, multiple of 256         */
    int blocks_per_sm;         /* resident blocks per SM of the persistent grid */
    int accum;                 /* gp_accum                                    */
    int long_edge;             /* compiled words; -1 no split, 1..255 split    */
    int long_rows_per_thread;  /* 4, 8 or 16 for the long bucket              */
    int long_blocks_per_sm;    /* resident blocks per SM of the long bucket   */
    int reserved[1];           /* must be 0                                   */
} gp_eval_opts;

/* ---- information ------------------------------------------------------- */
const char *gp_version(void);
const char *gp_status_string(int status);

/* ---- evaluation ---------------------------------------------------------
 * gp_evaluate: fitness of every program on rows [0, n_rows) (Sec. III-C3:
 * execution step fused with the loss and the weighted column reduction, so
 * the n_progs x n_rows prediction matrix is never stored).
 *   progs       [offsets[n_progs]] nodes; program p is
 *               progs[offsets[p] .. offsets[p+1]) in prefix order
 *   offsets     [n_progs + 1] int32, offsets[0] = 0, non-decreasing
 *   X           [n_feat][n_rows] float32, column-major (feature f's column
 *               starts at X + f * n_rows)
 *   y           [n_rows] float32 targets (labels 0/1 for GP_LOGLOSS)
 *   w           [n_rows] float32 weights, or NULL for all ones
 *   out_fitness [n_progs] float32; NaN for a malformed program
 * Batched persistent evaluator: one device pre-pass validates and compiles
 * all programs, sorts them by class (stack depth, extended functions) and
 * length, and one persistent launch per class works through (program,
 * row-chunk) items.  Scratch comes from a library-owned per-device cache
 * that grows on demand (cudaMalloc), so the first call at a new size
 * allocates; use gp_evaluate_ex with a caller workspace to avoid that (e.g.
 * under CUDA graph capture).  Every call that uses the cache on a device
 * shares it: calls that could overlap on the GPU (different streams, or
 * host threads without ordering) must be serialised by the caller, or each
 * given its own workspace.  The same inputs give bit-identical fitness on
 * every call. */
int gp_evaluate(const gp_node *progs, const int32_t *offsets, int n_progs,
                const float *X, int64_t n_rows, int n_feat, const float *y,
                const float *w, int metric, float *out_fitness, void *stream);

/* As gp_evaluate, with explicit tunables, optional FP64 fitness
 * (out_fitness64 [n_progs], may be NULL), optional per-program validator
 * status (out_prog_status [n_progs], may be NULL) and a caller workspace
 * `ws` of `ws_bytes` bytes (256-byte aligned, at least gp_workspace_size
 * bytes; ws == NULL uses the library cache).  With a caller workspace the
 * call performs no allocation and no synchronisation. */
int gp_evaluate_ex(const gp_node *progs, const int32_t *offsets, int n_progs,
                   const float *X, int64_t n_rows, int n_feat,
                   const float *y, const float *w, int metric,
                   const gp_eval_opts *opts, float *out_fitness,
                   double *out_fitness64, int32_t *out_prog_status, void *ws,
                   size_t ws_bytes, void *stream);

/* Bytes of workspace gp_evaluate_ex needs for this shape and these opts,
 * whatever the metric (GP_PEARSON needs the most: 24 more bytes per
 * program and row chunk). */
size_t gp_workspace_size(int n_progs, int64_t n_rows, int n_feat,
                         const gp_eval_opts *opts);

/* The tunables gp_evaluate_ex would use for this shape: `opts` (may be NULL)
 * with every zero field filled from the autotuner's record for the shape, or
 * else from the built-in defaults (rows_per_thread 4; chunk_rows sized for
 * about 16 work items per resident warp, 1024..16384 rows; blocks_per_sm 0 =
 * as many as fit).  Programs deeper than 8 stack slots, and programs that
 * use a function from GP_SQ on, always run with 4 rows per thread, whatever
 * rows_per_thread says.  Returns GP_ERR_ARG for invalid opts. */
int gp_resolve_opts(int n_progs, int64_t n_rows, int n_feat, const gp_eval_opts *opts,
                    gp_eval_opts *out);

/* Plain evaluator: one kernel launch per program, one row per thread in
 * blocks of 256 rows, programs read node by node from global memory and a
 * 20-slot stack held by predicated register selects (the shape of the
 * paper's execution kernel, Sec. III-C3 and III-D1), loss fused, per-block
 * partial sums reduced in FP64.  Same arguments and results as
 * gp_evaluate (fitness equal within the FP32 summation order) for the four
 * loss metrics; GP_PEARSON returns GP_ERR_ARG. */
int gp_evaluate_plain(const gp_node *progs, const int32_t *offsets,
                      int n_progs, const float *X, int64_t n_rows, int n_feat,
                      const float *y, const float *w, int metric,
                      float *out_fitness, void *stream);

/* Predictions (debug / parity path): out_pred [n_progs][n_rows] float32,
 * the value of program p on row i; NaN rows for a malformed program.  Uses
 * the same interpreter as gp_evaluate. */
int gp_predict(const gp_node *progs, const int32_t *offsets, int n_progs,
               const float *X, int64_t n_rows, int n_feat, float *out_pred,
               void *stream);

/* Predictions as gp_predict, with the evaluator's rows per thread taken
 * from opts (NULL: the defaults; only rows_per_thread is read, 4 or 8, and
 * it applies to the programs of the common class -- stack of at most 7
 * values, no extended function -- the others always run 4 rows per
 * thread).  Every prediction is the same bits whatever rows_per_thread
 * says: the per-row operations do not depend on how rows are grouped.
 * Returns GP_ERR_ARG for bad arguments or opts. */
int gp_predict_ex(const gp_node *progs, const int32_t *offsets, int n_progs,
                  const float *X, int64_t n_rows, int n_feat, const gp_eval_opts *opts,
                  float *out_pred, void *stream);

/* End-to-end variant of gp_evaluate for HOST buffers: progs, offsets, X,
 * y, w (may be NULL) and out_fitness are host pointers (pinned memory is
 * fastest).  Validates the programs on the host first (GP_ERR_PROGRAM,
 * nothing launched), copies the inputs to the device, evaluates, copies
 * the fitness back and synchronises `stream` before returning. */
int gp_evaluate_host(const gp_node *progs, const int32_t *offsets,
                     int n_progs, const float *X, int64_t n_rows, int n_feat,
                     const float *y, const float *w, int metric,
                     float *out_fitness, void *stream);

/* Host-side validation (no GPU needed).  progs/offsets are HOST pointers;
 * out_status [n_progs] receives gp_prog_status codes and out_high_water
 * [n_progs] (may be NULL) the largest stack height of the reverse scan
 * (a stack of 20 evaluates it iff <= 20, Sec. III-C2).  Returns GP_OK if
 * every program is valid, GP_ERR_PROGRAM otherwise, GP_ERR_ARG for bad
 * offsets. */
int gp_validate_host(const gp_node *progs, const int32_t *offsets,
                     int n_progs, int n_feat, int32_t *out_status,
                     int32_t *out_high_water);

/* ---- selection ----------------------------------------------------------
 * Tournament selection (Sec. III-C1): tournament t draws tourn_size program
 * indices with replacement from Philox4x32-10 (Salmon et al. 2011, cited
 * in Sec. III-B), key = (seed lo32, seed hi32), counter = (j / 4, t,
 * offset lo32, offset hi32), word j % 4, index = (u * n_progs) >> 32; the
 * winner is the draw with the strictly best adjusted fitness (ties: the
 * earliest draw; NaN is the worst), adjusted = raw + parsimony * len when
 * smaller is better, raw - parsimony * len otherwise (Eqs. parsimony,
 * fitness).  len = offsets[p+1] - offsets[p]; offsets may be NULL (no
 * penalty).  out_idx [n_tourn] int32.  One thread per tournament. */
int gp_tournament_ex(const float *fitness, const int32_t *offsets,
                     int n_progs, int n_tourn, int tourn_size,
                     float parsimony, int greater_is_better, uint64_t seed,
                     uint64_t offset, int32_t *out_idx, void *stream);

/* Short form: n_tourn = n_progs, no parsimony, smaller is better, offset
 * 0, legacy default stream. */
int gp_tournament(const float *fitness, int n_progs, int tourn_size,
                  uint64_t seed, int32_t *out_idx);

/* ---- mutation on the device ---------------------------------------------
 * Builds the next population from tournament winners on the GPU, so a whole
 * generation (evaluate, select, mutate) runs without a host round trip; the
 * paper mutates on the CPU (Sec. III-C2, III-D2) and names this as future
 * work (Sec. V).  Offspring t has parent parents[2t] and donor
 * parents[2t+1] (e.g. gp_tournament_ex with n_tourn = 2 n_out) and one
 * Philox4x32-10 stream: word k = Philox(counter = (k/4, t, offset lo32,
 * offset hi32), key = (seed lo32, seed hi32))[k % 4], taken in order; a word
 * u picks an index in [0, n) as (u n) >> 32 and a kind by comparing u with
 * the cumulative thresholds floor(p 2^32) (probabilities summed in double
 * in the order crossover, subtree, hoist, point).  Use another seed or
 * offset than the tournament's.
 *   crossover   node i of the parent and node j of the donor (uniform); the
 *               child is the parent with subtree i replaced by donor
 *               subtree j; while the child would exceed 255 nodes or 20
 *               stack slots, j moves to a node drawn uniformly among its
 *               proper descendants (the hoisted crossover of Sec. III-C2)
 *   subtree     a random grow tree of depth <= subtree_depth is the donor
 *               (drawn first), then as crossover from its root
 *   hoist       node i, then k among the proper descendants of i (k = i for
 *               a terminal); subtree i is replaced by subtree k
 *   point       each node in prefix order is replaced with probability
 *               p_point_replace: a function by an allowed function of the
 *               same arity, a terminal by a new terminal
 *   reproduction  the parent unchanged
 * A new terminal is variable f when a word picks f < n_feat in [0, n_feat],
 * else the constant (w >> 8) 2^-23 - 1 of the next word w.  A grow-tree
 * node above the depth limit is a terminal when a word picks one of 2
 * terminal kinds among 2 + (number of allowed functions), else an allowed
 * function (uniform).  A parent that is not a valid program is copied (the
 * one-node program 0 when its length is outside 1..255); an invalid donor
 * makes a crossover a reproduction; a parent index out of range gives the
 * program 0 and sets GP_DEV_BAD_PARENT. */
enum gp_mut_kind {
    GP_MUT_REPRODUCTION = 0, GP_MUT_CROSSOVER = 1, GP_MUT_SUBTREE = 2,
    GP_MUT_HOIST = 3, GP_MUT_POINT = 4
};

typedef struct gp_mut_params {
    float p_crossover;      /* probabilities of the kinds; reproduction    */
    float p_subtree;        /* takes the rest (their sum must be <= 1)     */
    float p_hoist;
    float p_point;
    float p_point_replace;  /* per-node replacement probability (point)    */
    int subtree_depth;      /* depth limit of subtree mutation's tree, 0..6 */
    uint32_t functions;     /* bit (1 << op) per function new nodes may use */
    int reserved[4];        /* must be 0                                   */
} gp_mut_params;

/* Bytes of scratch gp_mutate needs for n_out offspring. */
size_t gp_mutate_workspace_size(int n_out);

/* progs/offsets: the current population (n_progs programs, device);
 * parents [2 n_out] int32 (device); params (host); out_progs: capacity
 * n_out * 255 nodes (device); out_offsets [n_out + 1] (device, written by
 * the call: out_offsets[0] = 0); out_kind [n_out] (device, may be NULL):
 * the gp_mut_kind each offspring got.  ws: scratch of ws_bytes (256-byte
 * aligned, at least gp_mutate_workspace_size) or NULL for the library
 * cache.  1 <= n_out <= 2^22, 1 <= n_feat <= 32767.  Asynchronous;
 * GP_ERR_ARG for bad arguments (nothing launched). */
int gp_mutate(const gp_node *progs, const int32_t *offsets, int n_progs, int n_feat,
              const int32_t *parents, int n_out, const gp_mut_params *params,
              uint64_t seed, uint64_t offset, gp_node *out_progs,
              int32_t *out_offsets, int32_t *out_kind, void *ws, size_t ws_bytes,
              void *stream);

/* ---- constant tuning (no counterpart in the paper) ----------------------
 * Gradient of each program's fitness with respect to its ephemeral
 * constants, by a reverse-mode adjoint sweep per row that recomputes the
 * forward values instead of storing n_progs x n_rows x len of them.
 * Constant k of program p is its k-th CONST node in prefix order;
 * out_grad [n_progs][16] float32 (slots >= the program's constant count
 * are 0), out_fitness [n_progs] (may be NULL).  Derivatives of protected
 * operators are 0 on the protected branch; MAE uses sign(p - y) (0 at
 * equality); RMSE = MSE gradient / (2 RMSE) (0 when RMSE == 0).  A program
 * with more than 16 constants gets NaN gradients and sets
 * GP_DEV_TOO_MANY_CONSTS.  Loss metrics only (GP_PEARSON returns
 * GP_ERR_ARG).  Scratch as for gp_evaluate. */
int gp_const_grad(const gp_node *progs, const int32_t *offsets, int n_progs,
                  const float *X, int64_t n_rows, int n_feat, const float *y,
                  const float *w, int metric, float *out_grad,
                  float *out_fitness, void *stream);

/* One Adam step (Kingma & Ba 2015) on the constants, in place in `progs`:
 * with g = grad[p][k], m = beta1 m + (1-beta1) g, v = beta2 v + (1-beta2)
 * g^2, c -= lr * (m / (1-beta1^step)) / (sqrt(v / (1-beta2^step)) + eps).
 * m, v [n_progs][16] float32 state owned by the caller (zero before step
 * 1).  step >= 1.  A slot whose gradient is not finite keeps its constant
 * and its m, v unchanged. */
int gp_adam_step(gp_node *progs, const int32_t *offsets, int n_progs,
                 const float *grad, float *m, float *v, int step, float lr,
                 float beta1, float beta2, float eps, void *stream);

/* The constants of each program as a dense array, and back: constant k of
 * program p is its k-th CONST node in prefix order (the numbering of
 * gp_const_grad), stored at consts[p * 16 + k].  gp_get_consts writes all
 * 16 slots of every program (slots past its constant count are 0, a
 * malformed offset range leaves the whole row 0); gp_set_consts writes the
 * first min(count, 16) slots into the nodes' `c` fields in place and reads
 * nothing else.  Used to expose the constants as one tensor to automatic
 * differentiation. */
int gp_get_consts(const gp_node *progs, const int32_t *offsets, int n_progs,
                  float *out_consts, void *stream);
int gp_set_consts(gp_node *progs, const int32_t *offsets, int n_progs,
                  const float *consts, void *stream);

/* ---- runtime --------------------------------------------------------------
 * Synchronises `stream`, returns the device status bits accumulated since
 * the last call into *flags and clears them. */
int gp_last_device_status(void *stream, uint32_t *flags);

/* Searches the tunables of the batched evaluator on these inputs and
 * remembers the fastest for this problem shape; writes it to *best (may be
 * NULL).  Later calls with zero opts fields use it.  The search is staged:
 * rows_per_thread x chunk_rows, then blocks_per_sm, then the length-bucket
 * edge (none, 12, 16, 24, 32 compiled words) with the long bucket's rows per
 * thread, a split being taken only when it is at least 1% faster than one
 * launch; every candidate is timed as the median of three calls after one
 * warm-up (CUDA events on `stream`, synchronising), on the first 2^21 rows
 * when there are more.  GP_ERR_ARG for GP_SPEARMAN. */
int gp_autotune(const gp_node *progs, const int32_t *offsets, int n_progs,
                const float *X, int64_t n_rows, int n_feat, const float *y,
                const float *w, int metric, gp_eval_opts *best, void *stream);

/* Measurement only: sustained issue rates of the FP32 pipe (FADD) and of
 * the special-function unit per function, over all SMs, in lane-operations
 * per second, measured with CUDA events.  out[8]: out[0] = fp32 FADD,
 * out[1] = ex2, out[2] = rcp, out[3] = rsqrt, out[4] = lg2, out[5] = sin,
 * out[6] = SM count, out[7] = 0.  Synchronises. */
int gp_probe_pipes(double *out, void *stream);

/* Measurement only.  While enabled (on != 0), every batched evaluation
 * records a CUDA event pair on its stream around the evaluator's persistent
 * launches.  gp_timing_read waits for the recorded events, returns the sum
 * of their elapsed times in *total_ms and their count in *n_calls, and
 * forgets them.  Enabling or disabling also forgets them.  Do not enable
 * it while capturing a CUDA graph. */
int gp_timing_enable(int on);
int gp_timing_read(double *total_ms, int *n_calls);

/* ---- evaluation without allocation (no counterpart in the paper) --------
 * For callers that cannot allocate device memory at evaluation time: a
 * serving process whose device memory is handed out at start-up to another
 * allocator, code that must not call cudaMalloc/cudaFree because those can
 * synchronise the device, or a caller with no allocator of its own.
 * gp_evaluate_static takes gp_evaluate's arguments and, for the fused
 * metrics (GP_MAE ... GP_PEARSON), computes what gp_evaluate computes; it
 * returns GP_ERR_ARG for GP_SPEARMAN, whose scratch grows with the batch.
 * It uses a fixed scratch array of GP_STATIC_SCRATCH_BYTES that is part of
 * the library's device image, which every GPU that loads the library holds
 * until the process exits; it calls no allocating routine.  When the
 * workspace of the default tunables fits, the fitness is gp_evaluate's,
 * bit for bit.  When it does not, the call uses longer row chunks (65536
 * rows, then 4x longer each time) until it fits -- its fitness then equals
 * gp_evaluate_ex with the opts gp_static_opts reports, bit for bit, and
 * gp_evaluate's within the FP32 summation order; at P = 4096 programs and
 * 16M rows that is 65536-row chunks in about 12 MiB.  A problem that fits
 * with none gets GP_ERR_WORKSPACE and nothing is launched.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * and keeps it for the life of that device's context (gp_shutdown forgets
 * it), so make that first call before any stream capture.  All calls share
 * the one array and it keeps the last call's contents: calls that overlap
 * on the GPU (different streams, or host threads without ordering) race;
 * serialise them. */
#define GP_STATIC_SCRATCH_BYTES (16u << 20)
int gp_evaluate_static(const gp_node *progs, const int32_t *offsets,
                       int n_progs, const float *X, int64_t n_rows, int n_feat,
                       const float *y, const float *w, int metric,
                       float *out_fitness, void *stream);

/* The tunables gp_evaluate_static uses for this problem (chunk_rows 0: the
 * defaults; otherwise the longer row chunks it falls back to), without any
 * device work.  GP_ERR_WORKSPACE when no chunk length fits the array,
 * GP_ERR_ARG for bad arguments or GP_SPEARMAN. */
int gp_static_opts(int n_progs, int64_t n_rows, int n_feat, int metric,
                   gp_eval_opts *out);

/* Frees the library's cached device scratch on every device and forgets the
 * device addresses gp_evaluate_static looked up. */
void gp_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* GP_H_ */
