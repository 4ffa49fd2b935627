// gp_api.cu -- the C ABI of libgp (include/gp.h): argument checks, the
// per-device scratch cache, launch sequences, host-side validation, the
// host-buffer end-to-end path and the autotuner.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <cmath>
#include <mutex>
#include <tuple>
#include <vector>

#include "gp_internal.cuh"

using namespace gpk;

// Device status word: kernels OR problem bits into it; gp_last_device_status
// reads and clears it.  Host code reaches it through cudaGetSymbolAddress.
__device__ unsigned int g_gp_status_word;

namespace {

constexpr int kMaxDevices = 64;

struct ShapeKey {
    int n_progs;
    int64_t n_rows;
    int n_feat;
    bool operator<(const ShapeKey &o) const {
        return std::tie(n_progs, n_rows, n_feat) < std::tie(o.n_progs, o.n_rows, o.n_feat);
    }
};

struct DevCtx {
    bool init = false;
    int sms = 0;
    unsigned int *status = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *stage = nullptr;
    size_t stage_bytes = 0;
    void *rank = nullptr;  // Spearman: predictions, sort buffers, target ranks
    size_t rank_bytes = 0;
    std::map<ShapeKey, gp_eval_opts> tuned;
};

std::mutex g_mu;
DevCtx g_ctx[kMaxDevices];

// measurement hook (gp_timing_enable / gp_timing_read)
struct TimingState {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> live, pool;
};
TimingState g_timing;

std::pair<cudaEvent_t, cudaEvent_t> timing_pair() {
    std::lock_guard<std::mutex> g(g_mu);
    std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
    if (!g_timing.pool.empty()) {
        e = g_timing.pool.back();
        g_timing.pool.pop_back();
    } else {
        cudaEventCreate(&e.first);
        cudaEventCreate(&e.second);
    }
    g_timing.live.push_back(e);
    return e;
}

int ctx_of_current(DevCtx **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GP_ERR_CUDA;
    // the first call on a device fills its context; host threads may race here
    std::lock_guard<std::mutex> g(g_mu);
    DevCtx &c = g_ctx[dev];
    if (!c.init) {
        if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return GP_ERR_CUDA;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gp_status_word) != cudaSuccess) return GP_ERR_CUDA;
        c.status = static_cast<unsigned int *>(p);
        c.init = true;
    }
    *out = &c;
    return GP_OK;
}

// grow-only device buffer; the old one is freed (cudaFree synchronises)
int grow(void **ptr, size_t *cap, size_t need) {
    if (*cap >= need && *ptr) return GP_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    size_t want = std::max(need, (size_t)1 << 20);
    if (cudaMalloc(ptr, want) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return GP_ERR_NOMEM;
    }
    *cap = want;
    return GP_OK;
}

inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

#define GP_CUDA(x)                                    \
    do {                                              \
        if ((x) != cudaSuccess) {                     \
            cudaGetLastError();                       \
            return GP_ERR_CUDA;                       \
        }                                             \
    } while (0)

int check_common(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                 int64_t n_rows, int n_feat) {
    if (!progs || !offsets || !X) return GP_ERR_ARG;
    if (n_progs < 1 || n_rows < 1 || n_feat < 1 || n_feat > 32767) return GP_ERR_ARG;
    if (n_rows > ((int64_t)1 << 40)) return GP_ERR_ARG;
    return GP_OK;
}

// every metric of the batched evaluator
int check_metric(int metric) {
    return (metric >= GP_MAE && metric <= GP_SPEARMAN) ? GP_OK : GP_ERR_ARG;
}

// the metrics fused into the evaluator (no materialised predictions)
int check_fused_metric(int metric) {
    return (metric >= GP_MAE && metric <= GP_PEARSON) ? GP_OK : GP_ERR_ARG;
}

// the per-row loss metrics (plain evaluator, constant gradients)
int check_loss_metric(int metric) {
    return (metric >= GP_MAE && metric <= GP_LOGLOSS) ? GP_OK : GP_ERR_ARG;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ---- tunables -----------------------------------------------------------
int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// L2 share for one row chunk of every column (the blocks resident at any
// moment work on one or two chunks; the L2 holds 129 MB)
constexpr int64_t kChunkL2Bytes = 48ll << 20;

int64_t default_chunk(int n_progs, int64_t n_rows, int n_feat, int sms, int64_t pass_rows = 1024) {
    // enough items for dynamic balancing (about 16 per resident warp),
    // chunks of at most 16K rows (measured on Pagie-1 x 4096 programs at
    // 1M and 16M rows: 16K-row chunks beat 64K by 4%, 8K and 32K by 1%),
    // and for wide tables few enough rows that one chunk of all columns
    // stays in L2
    const double items_wanted = 16.0 * sms * 24.0;
    int64_t c = (int64_t)((double)n_rows * (double)n_progs / items_wanted);
    c = std::min<int64_t>(c, 16384);
    c = std::min<int64_t>(c, kChunkL2Bytes / (4 * ((int64_t)n_feat + 2)));
    // whole passes of a block (8 warps x 32 lanes x 4 rows, or 8 rows:
    // pass_rows): a partial last pass idles warps (measured on 500K x 2000:
    // 6400-row chunks 5% slower than 6144)
    c = std::max<int64_t>(c / pass_rows * pass_rows, pass_rows);
    return std::min<int64_t>(c, round_up(n_rows, 256));
}

int resolve_opts(const gp_eval_opts *in, int n_progs, int64_t n_rows, int n_feat, DevCtx *c,
                 gp_eval_opts *out) {
    gp_eval_opts o{};
    if (in) o = *in;
    if (o.reserved[0] != 0) return GP_ERR_ARG;
    if (o.rows_per_thread == 0 || o.chunk_rows == 0 || o.blocks_per_sm == 0 || o.long_edge == 0) {
        std::lock_guard<std::mutex> g(g_mu);
        auto it = c->tuned.find(ShapeKey{n_progs, n_rows, n_feat});
        if (it != c->tuned.end()) {
            if (o.rows_per_thread == 0) o.rows_per_thread = it->second.rows_per_thread;
            if (o.chunk_rows == 0) o.chunk_rows = it->second.chunk_rows;
            if (o.blocks_per_sm == 0) o.blocks_per_sm = it->second.blocks_per_sm;
            if (o.long_edge == 0) {
                o.long_edge = it->second.long_edge;
                o.long_rows_per_thread = it->second.long_rows_per_thread;
                o.long_blocks_per_sm = it->second.long_blocks_per_sm;
            }
        }
    }
    // length buckets: none unless asked for or tuned
    if (o.long_edge == 0) o.long_edge = -1;
    if (o.long_edge != -1 && (o.long_edge < 1 || o.long_edge > 255)) return GP_ERR_ARG;
    // 8 rows per thread: 64 registers, 4 blocks (32 warps) per SM, measured
    // 5% faster than 4 rows (48 registers, 5 blocks) on Pagie-1 16M x 4096
    // with RMSE, 0.5% with Pearson; the autotuner picks it on every
    // benchmark workload
    if (o.rows_per_thread == 0) o.rows_per_thread = 8;
    if (o.rows_per_thread != 4 && o.rows_per_thread != 8 && o.rows_per_thread != 16)
        return GP_ERR_ARG;
    if (o.chunk_rows == 0)
        o.chunk_rows = (int)default_chunk(n_progs, n_rows, n_feat, c->sms,
                                          o.rows_per_thread == 4 ? 1024 : 2048);
    if (o.chunk_rows < 256 || o.chunk_rows % 256 != 0) return GP_ERR_ARG;
    if (o.blocks_per_sm < 0 || o.blocks_per_sm > 32) return GP_ERR_ARG;
    if (o.accum != GP_ACCUM_FP64 && o.accum != GP_ACCUM_KAHAN32) return GP_ERR_ARG;
    if (o.long_rows_per_thread == 0) o.long_rows_per_thread = o.rows_per_thread;
    if (o.long_rows_per_thread != 4 && o.long_rows_per_thread != 8 && o.long_rows_per_thread != 16)
        return GP_ERR_ARG;
    if (o.long_blocks_per_sm < 0 || o.long_blocks_per_sm > 32) return GP_ERR_ARG;
    *out = o;
    return GP_OK;
}

int eval_info(int rpt, int fmode, int cls, int block, int *regs, bool mom = false,
              bool pred = false) {
    if (rpt == 4) return fmode == 2 ? info_eval_r4_f2(cls, block, regs, mom) : info_eval_r4_f0(cls, block, regs, mom);
    if (rpt == 8)
        return fmode == 2 ? info_eval_r8_f2(cls, block, regs, mom, pred)
                          : info_eval_r8_f0(cls, block, regs, mom, pred);
    return fmode == 2 ? info_eval_r16_f2(cls, block, regs, mom) : info_eval_r16_f0(cls, block, regs, mom);
}

cudaError_t eval_launch(const EvalArgs &a, int rpt, int fmode, int grid, int block, cudaStream_t st) {
    if (rpt == 4) return fmode == 2 ? launch_eval_r4_f2(a, grid, block, st) : launch_eval_r4_f0(a, grid, block, st);
    if (rpt == 8) return fmode == 2 ? launch_eval_r8_f2(a, grid, block, st) : launch_eval_r8_f0(a, grid, block, st);
    return fmode == 2 ? launch_eval_r16_f2(a, grid, block, st) : launch_eval_r16_f0(a, grid, block, st);
}

struct Plan {
    gp_eval_opts o;
    int n_chunks;
    Layout L;
};

// moments: the workspace also holds the correlation extras
int make_plan(const gp_eval_opts *opts, int n_progs, int64_t n_rows, int n_feat, DevCtx *c,
              Plan *pl, bool moments) {
    int rc = resolve_opts(opts, n_progs, n_rows, n_feat, c, &pl->o);
    if (rc) return rc;
    pl->n_chunks = (int)((n_rows + pl->o.chunk_rows - 1) / pl->o.chunk_rows);
    pl->L = make_layout(n_progs, pl->n_chunks, false, moments);
    return GP_OK;
}

// the batched evaluation sequence on a carved workspace
// ld: the column stride of X (n_rows, or more when the rows are a prefix)
int run_evaluate(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                 int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                 const Plan &pl, const Workspace &W, DevCtx *c, float *out, double *out64,
                 int32_t *out_status, cudaStream_t st, int64_t ld = -1) {
    if (ld < 0) ld = n_rows;
    const bool mom = metric == GP_PEARSON;
    GP_CUDA(cudaMemsetAsync(W.counters, 0, 8 * sizeof(unsigned long long), st));
    CompileArgs ca{progs, offsets, n_progs, n_feat, W.code, W.meta,
                   c->status, nullptr};
    if (mom) {
        ca.X = X;
        ca.ld = ld;
        ca.shift = W.shift;
    }
    GP_CUDA(launch_compile(ca, st));
    const bool split = pl.o.long_edge > 0;
    GP_CUDA(launch_order(W.meta, n_progs, W.order, W.class_count, st, 0, split ? pl.o.long_edge : 0));
    GP_CUDA(launch_sumw(w, n_rows, W.sumw_part, W.sumw, st));
    if (mom) GP_CUDA(launch_ystats(y, w, n_rows, W.sumw, W.ystat_part, W.ystat, st));
    const int fmode = (n_feat <= 2) ? 2 : 0;
    // the moment epilogue has instances for 4 and 8 rows per thread
    const int rpt = (mom && pl.o.rows_per_thread == 16) ? 8 : pl.o.rows_per_thread;
    const bool vec = aligned16(X) && aligned16(y) && (!w || aligned16(w)) && (n_rows % 4 == 0) &&
                     (ld % 4 == 0);
    std::pair<cudaEvent_t, cudaEvent_t> tev{nullptr, nullptr};
    if (g_timing.on) {
        tev = timing_pair();
        GP_CUDA(cudaEventRecord(tev.first, st));
    }
    // launches: class 0 (or, split by length, its long then its short
    // programs), classes 1, 2 and 3
    for (int launch = split ? -1 : 0; launch < kNumClasses; ++launch) {
        const int cls = launch < 0 ? 0 : launch;
        EvalArgs ea{};
        ea.code = W.code;
        ea.meta = W.meta;
        ea.order = W.order;
        ea.class_count = W.class_count;
        ea.cls = cls;
        ea.X = X;
        ea.ld = (fmode == 2) ? (n_feat == 2 ? ld : 0) : ld;
        ea.n_rows = n_rows;
        ea.y = y;
        ea.w = w;
        ea.n_progs = n_progs;
        ea.metric = metric;
        ea.chunk_rows = pl.o.chunk_rows;
        ea.n_chunks = pl.n_chunks;
        ea.sub = split && cls == kClassShallow ? (launch < 0 ? 1 : 2) : 0;
        ea.counter = W.counters + (ea.sub == 1 ? kNumClasses : cls);
        ea.part = W.part;
        ea.dev_status = c->status;
        ea.vec_ok = vec ? 1 : 0;
        if (mom) {
            ea.mom = W.mom;
            ea.shift = W.shift;
            ea.ystat = W.ystat;
        }
        // classes 1-3 keep 4 rows per thread (the 19-slot stack would
        // otherwise leave room for one block per SM; classes 2 and 3 are
        // rare); the same chunk partition serves all four
        const int rpt_long = (mom && pl.o.long_rows_per_thread == 16) ? 8 : pl.o.long_rows_per_thread;
        const int rpt_c = (cls == kClassShallow) ? (ea.sub == 1 ? rpt_long : rpt) : 4;
        const int want = ea.sub == 1 ? pl.o.long_blocks_per_sm : pl.o.blocks_per_sm;
        const int block = kEvalBlockThreads;
        int occ = eval_info(rpt_c, fmode, cls, block, nullptr, mom);
        if (occ < 1) occ = 1;
        int bps = want > 0 ? std::min(want, occ) : occ;
        GP_CUDA(eval_launch(ea, rpt_c, fmode, c->sms * bps, block, st));
    }
    if (tev.second) GP_CUDA(cudaEventRecord(tev.second, st));
    FinalizeArgs fa{};
    fa.part = W.part;
    fa.mom = mom ? W.mom : nullptr;
    fa.ystat = mom ? W.ystat : nullptr;
    fa.n_chunks = pl.n_chunks;
    fa.n_progs = n_progs;
    fa.meta = W.meta;
    fa.sumw = W.sumw;
    fa.metric = metric;
    fa.accum = pl.o.accum;
    fa.out = out;
    fa.out64 = out64;
    fa.out_prog_status = out_status;
    GP_CUDA(launch_finalize(fa, st));
    return GP_OK;
}

int validate_one_host(const gp_node *p, int len, int n_feat, int *hw_out) {
    int sp = 0, hw = 0;
    *hw_out = 0;
    if (len < 1 || len > GP_MAX_LEN) return GP_PROG_BAD_LENGTH;
    for (int j = len - 1; j >= 0; --j) {
        const int op = p[j].op;
        int ar;
        if (op == GP_CONST || op == GP_VAR) ar = 0;
        else if ((op >= GP_ADD && op <= GP_DIV) || op == GP_MAX || op == GP_MIN) ar = 2;
        else if (op >= GP_SQRT && op <= GP_COSH) ar = 1;
        else return GP_PROG_BAD_OP;
        if (op == GP_VAR && (p[j].feat < 0 || p[j].feat >= n_feat)) return GP_PROG_BAD_FEATURE;
        if (ar == 0) ++sp;
        else {
            if (sp < ar) return GP_PROG_UNDERFLOW;
            sp -= ar - 1;
        }
        hw = std::max(hw, sp);
    }
    *hw_out = hw;
    if (sp != 1) return GP_PROG_LEFTOVER;
    if (hw > GP_MAX_STACK) return GP_PROG_TOO_DEEP;
    return GP_PROG_OK;
}

// predictions of programs [p0, p0 + b) whose compiled code and metadata
// are already in W (indexed by program id) into pred [b][n_rows]
int run_predict_compiled(const Workspace &W, int p0, int b, const float *X, int64_t n_rows,
                         int n_feat, float *out_pred, DevCtx *c, cudaStream_t st, int rpt = 4) {
    const int64_t chunk = std::min<int64_t>(round_up(n_rows, 256), 4096);
    const int n_chunks = (int)((n_rows + chunk - 1) / chunk);
    GP_CUDA(cudaMemsetAsync(W.counters, 0, 8 * sizeof(unsigned long long), st));
    GP_CUDA(launch_order(W.meta + p0, b, W.order, W.class_count, st));
    const bool vec = aligned16(X) && (n_rows % 4 == 0);
    const int fmode = (n_feat <= 2) ? 2 : 0;
    for (int cls = 0; cls < kNumClasses; ++cls) {
        EvalArgs ea{};
        ea.code = W.code + (size_t)p0 * kCodeStride;
        ea.meta = W.meta + p0;
        ea.order = W.order;
        ea.class_count = W.class_count;
        ea.cls = cls;
        ea.X = X;
        ea.ld = (fmode == 2) ? (n_feat == 2 ? n_rows : 0) : n_rows;
        ea.n_rows = n_rows;
        ea.n_progs = b;
        ea.metric = GP_MSE;
        ea.chunk_rows = chunk;
        ea.n_chunks = n_chunks;
        ea.counter = W.counters + cls;
        ea.pred = out_pred;
        ea.dev_status = c->status;
        ea.vec_ok = vec ? 1 : 0;
        if (cls == kClassShallow && rpt == 8) {
            // the class-0 instance at 8 rows per thread (its store epilogue)
            const int occ = eval_info(8, fmode, cls, kEvalBlockThreads, nullptr, false, true);
            GP_CUDA(eval_launch(ea, 8, fmode, c->sms * std::max(occ, 1), kEvalBlockThreads, st));
            continue;
        }
        const int occ = fmode == 2 ? info_predict_f2(cls, kEvalBlockThreads, nullptr)
                                   : info_predict(cls, kEvalBlockThreads, nullptr);
        const int grid = c->sms * std::max(occ, 1);
        GP_CUDA(fmode == 2 ? launch_predict_f2(ea, grid, kEvalBlockThreads, st)
                           : launch_predict(ea, grid, kEvalBlockThreads, st));
    }
    return GP_OK;
}

// the pre-pass of every program into the context's workspace (code, meta,
// order for up to n_progs programs); *W receives the carved workspace
int compile_all(const gp_node *progs, const int32_t *offsets, int n_progs, int n_feat,
                int32_t *out_status, DevCtx *c, Workspace *W, cudaStream_t st) {
    int rc;
    Layout L = make_layout(n_progs, 1, false);
    {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->ws, &c->ws_bytes, L.total))) return rc;
    }
    *W = carve(c->ws, L, false);
    CompileArgs ca{progs, offsets, n_progs, n_feat, W->code, W->meta,
                   c->status, out_status};
    GP_CUDA(launch_compile(ca, st));
    return GP_OK;
}

// every program's value on every row into pred [n_progs][n_rows]
int run_predict(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                int64_t n_rows, int n_feat, float *out_pred, int32_t *out_status, DevCtx *c,
                cudaStream_t st, int rpt = 4) {
    Workspace W;
    int rc = compile_all(progs, offsets, n_progs, n_feat, out_status, c, &W, st);
    if (rc) return rc;
    return run_predict_compiled(W, 0, n_progs, X, n_rows, n_feat, out_pred, c, st, rpt);
}

// Spearman: the target's ranks once, then batches of programs predicted
// into [B][N] (B chosen so the batch and its sort buffers take <= 2 GB),
// ranked and reduced
constexpr size_t kRankBudget = 2ull << 30;

int run_spearman(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                 int64_t n_rows, int n_feat, const float *y, const float *w, float *out,
                 double *out64, int32_t *out_status, DevCtx *c, cudaStream_t st) {
    if (n_rows >= ((int64_t)1 << 31) - 2) return GP_ERR_ARG;
    const int64_t per_prog = n_rows * 4 * 6;  // prediction, 4 sort arrays, slack
    int B = (int)std::max<int64_t>(1, std::min<int64_t>(n_progs, (int64_t)kRankBudget / per_prog));
    const size_t b_pred = (size_t)round_up((int64_t)B * n_rows * 4, 256);
    const size_t b_r2y = (size_t)round_up(n_rows * 4, 256);
    const size_t b_tp = (size_t)round_up((int64_t)target_part_bytes(n_rows), 256);
    const size_t b_scr = rank_scratch_bytes(B, n_rows);
    int rc;
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->rank, &c->rank_bytes, b_pred + b_r2y + b_tp + b_scr))) return rc;
        base = static_cast<char *>(c->rank);
    }
    float *pred = reinterpret_cast<float *>(base);
    uint32_t *r2y = reinterpret_cast<uint32_t *>(base + b_pred);
    double *tpart = reinterpret_cast<double *>(base + b_pred + b_r2y);
    void *scr = base + b_pred + b_r2y + b_tp;
    GP_CUDA(target_ranks(y, w, n_rows, scr, r2y, tpart, st));
    // the pre-pass once for all programs (one thread per program: compiled
    // batch by batch, its latency came back with every batch)
    Workspace W;
    if ((rc = compile_all(progs, offsets, n_progs, n_feat, out_status, c, &W, st))) return rc;
    for (int p0 = 0; p0 < n_progs; p0 += B) {
        const int b = std::min(B, n_progs - p0);
        if ((rc = run_predict_compiled(W, p0, b, X, n_rows, n_feat, pred, c, st))) return rc;
        GP_CUDA(spearman_batch(pred, b, n_rows, r2y, tpart, w, scr, out + p0,
                               out64 ? out64 + p0 : nullptr, st));
    }
    return GP_OK;
}

}  // namespace

namespace gpk {
// workspace bytes of one evaluation with this metric (0 for bad arguments)
size_t workspace_bytes_for(int n_progs, int64_t n_rows, int n_feat, const gp_eval_opts *opts,
                           int metric) {
    if (n_progs < 1 || n_rows < 1 || n_feat < 1 || check_fused_metric(metric)) return 0;
    DevCtx *c = nullptr;
    if (ctx_of_current(&c)) return 0;
    Plan pl;
    if (make_plan(opts, n_progs, n_rows, n_feat, c, &pl, metric == GP_PEARSON)) return 0;
    return pl.L.total;
}
}  // namespace gpk

extern "C" {

const char *gp_version(void) { return "libgp 1.0 (sm_103a)"; }

const char *gp_status_string(int s) {
    switch (s) {
    case GP_OK: return "ok";
    case GP_ERR_ARG: return "bad argument";
    case GP_ERR_PROGRAM: return "malformed program";
    case GP_ERR_CONSTS: return "more than 16 constants in a program";
    case GP_ERR_CUDA: return "CUDA runtime error";
    case GP_ERR_TIMEOUT: return "device loop cap reached";
    case GP_ERR_NOMEM: return "device allocation failed";
    case GP_ERR_WORKSPACE: return "workspace too small or misaligned";
    }
    return "unknown status";
}

size_t gp_workspace_size(int n_progs, int64_t n_rows, int n_feat, const gp_eval_opts *opts) {
    if (n_progs < 1 || n_rows < 1 || n_feat < 1) return 0;
    DevCtx *c = nullptr;
    if (ctx_of_current(&c)) return 0;
    Plan pl;
    if (make_plan(opts, n_progs, n_rows, n_feat, c, &pl, true)) return 0;
    return pl.L.total;
}


int gp_resolve_opts(int n_progs, int64_t n_rows, int n_feat, const gp_eval_opts *opts,
                    gp_eval_opts *out) {
    if (n_progs < 1 || n_rows < 1 || n_feat < 1 || !out) return GP_ERR_ARG;
    DevCtx *c = nullptr;
    int rc = ctx_of_current(&c);
    if (rc) return rc;
    Plan pl;
    if ((rc = make_plan(opts, n_progs, n_rows, n_feat, c, &pl, false))) return rc;
    *out = pl.o;
    return GP_OK;
}

int gp_evaluate_ex(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                   int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                   const gp_eval_opts *opts, float *out_fitness, double *out_fitness64,
                   int32_t *out_prog_status, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!y || !out_fitness) return GP_ERR_ARG;
    if ((rc = check_metric(metric))) return rc;
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    if (metric == GP_SPEARMAN) {  // library scratch only: its size depends on the batch
        if (ws) return GP_ERR_ARG;
        return run_spearman(progs, offsets, n_progs, X, n_rows, n_feat, y, w, out_fitness,
                            out_fitness64, out_prog_status, c, S(stream));
    }
    Plan pl;
    if ((rc = make_plan(opts, n_progs, n_rows, n_feat, c, &pl, metric == GP_PEARSON))) return rc;
    void *base = ws;
    if (ws) {
        if (ws_bytes < pl.L.total || ((uintptr_t)ws & 255u)) return GP_ERR_WORKSPACE;
    } else {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->ws, &c->ws_bytes, pl.L.total))) return rc;
        base = c->ws;
    }
    Workspace W = carve(base, pl.L, false);
    return run_evaluate(progs, offsets, n_progs, X, n_rows, n_feat, y, w, metric, pl, W, c,
                        out_fitness, out_fitness64, out_prog_status, S(stream));
}

int gp_evaluate(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                float *out_fitness, void *stream) {
    return gp_evaluate_ex(progs, offsets, n_progs, X, n_rows, n_feat, y, w, metric, nullptr,
                          out_fitness, nullptr, nullptr, nullptr, 0, stream);
}

int gp_evaluate_plain(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                      int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                      float *out_fitness, void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!y || !out_fitness) return GP_ERR_ARG;
    if ((rc = check_loss_metric(metric))) return rc;
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    const int64_t nb64 = (n_rows + 255) / 256;
    if (nb64 > (1 << 30)) return GP_ERR_ARG;
    const int n_blocks = (int)nb64;
    Layout L = make_layout(n_progs, n_blocks, false);
    {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->ws, &c->ws_bytes, L.total))) return rc;
    }
    Workspace W = carve(c->ws, L, false);
    cudaStream_t st = S(stream);
    CompileArgs ca{progs, offsets, n_progs, n_feat, W.code, W.meta,
                   c->status, nullptr};
    GP_CUDA(launch_compile(ca, st));
    GP_CUDA(launch_sumw(w, n_rows, W.sumw_part, W.sumw, st));
    PlainArgs pa{progs, offsets, W.meta, X, n_rows, n_rows, y, w, metric, n_blocks, W.part};
    for (int p = 0; p < n_progs; ++p) GP_CUDA(launch_plain(pa, p, st));
    FinalizeArgs fa{};
    fa.part = W.part;
    fa.n_chunks = n_blocks;
    fa.n_progs = n_progs;
    fa.meta = W.meta;
    fa.sumw = W.sumw;
    fa.metric = metric;
    fa.accum = GP_ACCUM_FP64;
    fa.out = out_fitness;
    GP_CUDA(launch_finalize(fa, st));
    return GP_OK;
}

int gp_predict(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
               int64_t n_rows, int n_feat, float *out_pred, void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!out_pred) return GP_ERR_ARG;
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    return run_predict(progs, offsets, n_progs, X, n_rows, n_feat, out_pred, nullptr, c, S(stream));
}

int gp_predict_ex(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                  int64_t n_rows, int n_feat, const gp_eval_opts *opts, float *out_pred,
                  void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!out_pred) return GP_ERR_ARG;
    const int rpt = opts && opts->rows_per_thread ? opts->rows_per_thread : 4;
    if (rpt != 4 && rpt != 8) return GP_ERR_ARG;
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    return run_predict(progs, offsets, n_progs, X, n_rows, n_feat, out_pred, nullptr, c,
                       S(stream), rpt);
}

int gp_validate_host(const gp_node *progs, const int32_t *offsets, int n_progs, int n_feat,
                     int32_t *out_status, int32_t *out_high_water) {
    if (!progs || !offsets || !out_status || n_progs < 1 || n_feat < 1) return GP_ERR_ARG;
    if (offsets[0] != 0) return GP_ERR_ARG;
    int rc = GP_OK;
    for (int p = 0; p < n_progs; ++p) {
        const int len = offsets[p + 1] - offsets[p];
        int hw = 0;
        const int s = (len < 0) ? GP_PROG_BAD_LENGTH : validate_one_host(progs + offsets[p], len, n_feat, &hw);
        out_status[p] = s;
        if (out_high_water) out_high_water[p] = hw;
        if (s != GP_PROG_OK) rc = GP_ERR_PROGRAM;
        if (len < 0) return GP_ERR_ARG;
    }
    return rc;
}

int gp_evaluate_host(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                     int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                     float *out_fitness, void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!y || !out_fitness) return GP_ERR_ARG;
    if ((rc = check_metric(metric))) return rc;
    if (offsets[0] != 0) return GP_ERR_ARG;
    for (int p = 0; p < n_progs; ++p) {
        int hw = 0;
        const int len = offsets[p + 1] - offsets[p];
        if (len < 0) return GP_ERR_ARG;
        if (validate_one_host(progs + offsets[p], len, n_feat, &hw) != GP_PROG_OK) return GP_ERR_PROGRAM;
    }
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    const size_t n_nodes = (size_t)offsets[n_progs];
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_nodes = al(n_nodes * sizeof(gp_node) + 8);
    const size_t b_off = al((size_t)(n_progs + 1) * sizeof(int32_t));
    const size_t b_X = al((size_t)n_feat * (size_t)n_rows * sizeof(float));
    const size_t b_y = al((size_t)n_rows * sizeof(float));
    const size_t b_w = w ? b_y : 0;
    const size_t b_out = al((size_t)n_progs * sizeof(float));
    const size_t need = b_nodes + b_off + b_X + b_y + b_w + b_out;
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->stage, &c->stage_bytes, need))) return rc;
        base = static_cast<char *>(c->stage);
    }
    gp_node *d_nodes = reinterpret_cast<gp_node *>(base);
    int32_t *d_off = reinterpret_cast<int32_t *>(base + b_nodes);
    float *d_X = reinterpret_cast<float *>(base + b_nodes + b_off);
    float *d_y = reinterpret_cast<float *>(base + b_nodes + b_off + b_X);
    float *d_w = w ? reinterpret_cast<float *>(base + b_nodes + b_off + b_X + b_y) : nullptr;
    float *d_out = reinterpret_cast<float *>(base + b_nodes + b_off + b_X + b_y + b_w);
    cudaStream_t st = S(stream);
    GP_CUDA(cudaMemcpyAsync(d_nodes, progs, n_nodes * sizeof(gp_node), cudaMemcpyHostToDevice, st));
    GP_CUDA(cudaMemcpyAsync(d_off, offsets, (size_t)(n_progs + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    GP_CUDA(cudaMemcpyAsync(d_X, X, (size_t)n_feat * n_rows * sizeof(float), cudaMemcpyHostToDevice, st));
    GP_CUDA(cudaMemcpyAsync(d_y, y, (size_t)n_rows * sizeof(float), cudaMemcpyHostToDevice, st));
    if (w) GP_CUDA(cudaMemcpyAsync(d_w, w, (size_t)n_rows * sizeof(float), cudaMemcpyHostToDevice, st));
    rc = gp_evaluate(d_nodes, d_off, n_progs, d_X, n_rows, n_feat, d_y, d_w, metric, d_out, stream);
    if (rc) return rc;
    GP_CUDA(cudaMemcpyAsync(out_fitness, d_out, (size_t)n_progs * sizeof(float), cudaMemcpyDeviceToHost, st));
    GP_CUDA(cudaStreamSynchronize(st));
    return GP_OK;
}

int gp_tournament_ex(const float *fitness, const int32_t *offsets, int n_progs, int n_tourn,
                     int tourn_size, float parsimony, int greater_is_better, uint64_t seed,
                     uint64_t offset, int32_t *out_idx, void *stream) {
    if (!fitness || !out_idx || n_progs < 1 || n_tourn < 0 || tourn_size < 1) return GP_ERR_ARG;
    TournArgs a{fitness, offsets, n_progs, n_tourn, tourn_size, parsimony,
                greater_is_better ? 1 : 0, seed, offset, out_idx};
    GP_CUDA(launch_tournament(a, S(stream)));
    return GP_OK;
}

int gp_tournament(const float *fitness, int n_progs, int tourn_size, uint64_t seed, int32_t *out_idx) {
    return gp_tournament_ex(fitness, nullptr, n_progs, n_progs, tourn_size, 0.0f, 0, seed, 0,
                            out_idx, nullptr);
}

int gp_const_grad(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                  int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                  float *out_grad, float *out_fitness, void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!y || !out_grad) return GP_ERR_ARG;
    if ((rc = check_loss_metric(metric))) return rc;
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    const int64_t chunk = default_chunk(n_progs, n_rows, n_feat, c->sms);
    const int n_chunks = (int)((n_rows + chunk - 1) / chunk);
    Layout L = make_layout(n_progs, n_chunks, true);
    {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->ws, &c->ws_bytes, L.total))) return rc;
    }
    Workspace W = carve(c->ws, L, true);
    cudaStream_t st = S(stream);
    GP_CUDA(cudaMemsetAsync(W.counters, 0, 8 * sizeof(unsigned long long), st));
    CompileArgs ca{progs, offsets, n_progs, n_feat, W.code, W.meta,
                   c->status, nullptr};
    ca.grad = 1;  // the gradient form: no constant folding, marker words
    GP_CUDA(launch_compile(ca, st));
    GP_CUDA(launch_order(W.meta, n_progs, W.order, W.class_count, st, 1));
    GP_CUDA(launch_sumw(w, n_rows, W.sumw_part, W.sumw, st));
    // one launch per bucket (constants, stack depth) of the compiled programs
    const bool vec = aligned16(X) && aligned16(y) && (!w || aligned16(w)) && (n_rows % 4 == 0) &&
                     (chunk % 4 == 0);
    for (int bucket = 0; bucket < kGradBuckets; ++bucket) {
        GradArgs ga{};
        ga.code = W.code;
        ga.meta = W.meta;
        ga.order = W.order;
        ga.class_count = W.class_count;
        ga.bucket = bucket;
        ga.X = X;
        ga.ld = n_rows;
        ga.n_rows = n_rows;
        ga.n_feat = n_feat;
        ga.y = y;
        ga.w = w;
        ga.metric = metric;
        ga.chunk_rows = chunk;
        ga.n_chunks = n_chunks;
        ga.counter = W.counters;
        ga.part = W.part;
        ga.gpart = W.gpart;
        ga.dev_status = c->status;
        ga.vec_ok = vec ? 1 : 0;
        GP_CUDA(launch_grad(ga, c->sms, st));
    }
    // the programs without constants: their loss partials from the
    // evaluator (no tangents; their gradient slots are 0)
    {
        EvalArgs ea{};
        ea.code = W.code;
        ea.code_stride = kGradCodeStride;
        ea.meta = W.meta;
        ea.order = W.order;
        ea.class_count = W.class_count;
        // compiled stacks of up to kSmallDepth values: the 7-slot instance
        ea.cls = kClassShallow8;
        ea.qcls = kGradBuckets + 1;
        ea.X = X;
        ea.ld = n_rows;
        ea.n_rows = n_rows;
        ea.y = y;
        ea.w = w;
        ea.n_progs = n_progs;
        ea.metric = metric;
        ea.chunk_rows = chunk;
        ea.n_chunks = n_chunks;
        ea.counter = W.counters + kGradBuckets;
        ea.part = W.part;
        ea.dev_status = c->status;
        ea.vec_ok = vec ? 1 : 0;
        const int fmode = (n_feat <= 2) ? 2 : 0;
        const int occ = eval_info(4, fmode, kClassShallow8, kEvalBlockThreads, nullptr);
        GP_CUDA(eval_launch(ea, 4, fmode, c->sms * std::max(occ, 1), kEvalBlockThreads, st));
    }
    GradFinalizeArgs fa{W.part, W.gpart, n_chunks, n_progs, W.meta, W.sumw, metric,
                        out_grad, out_fitness};
    GP_CUDA(launch_grad_finalize(fa, st));
    return GP_OK;
}

int gp_adam_step(gp_node *progs, const int32_t *offsets, int n_progs, const float *grad, float *m,
                 float *v, int step, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!progs || !offsets || !grad || !m || !v || n_progs < 1 || step < 1) return GP_ERR_ARG;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f))
        return GP_ERR_ARG;
    AdamArgs a{progs, offsets, nullptr, n_progs, grad, m, v, step, lr, beta1, beta2, eps};
    GP_CUDA(launch_adam(a, S(stream)));
    return GP_OK;
}

size_t gp_mutate_workspace_size(int n_out) {
    if (n_out < 1 || n_out > (1 << 22)) return 0;
    return round_up((int64_t)n_out * 256 * (int64_t)sizeof(gp_node), 256) +
           round_up((int64_t)n_out * (int64_t)sizeof(int32_t), 256);
}

int gp_mutate(const gp_node *progs, const int32_t *offsets, int n_progs, int n_feat,
              const int32_t *parents, int n_out, const gp_mut_params *params, uint64_t seed,
              uint64_t offset, gp_node *out_progs, int32_t *out_offsets, int32_t *out_kind,
              void *ws, size_t ws_bytes, void *stream) {
    if (!progs || !offsets || !parents || !params || !out_progs || !out_offsets) return GP_ERR_ARG;
    if (n_progs < 1 || n_feat < 1 || n_feat > 32767 || n_out < 1 || n_out > (1 << 22))
        return GP_ERR_ARG;
    const gp_mut_params &q = *params;
    for (int i = 0; i < 4; ++i)
        if (q.reserved[i] != 0) return GP_ERR_ARG;
    const float pk[4] = {q.p_crossover, q.p_subtree, q.p_hoist, q.p_point};
    MutArgs a{};
    double cum = 0.0;
    for (int i = 0; i < 4; ++i) {
        if (!(pk[i] >= 0.0f && pk[i] <= 1.0f)) return GP_ERR_ARG;
        cum += (double)pk[i];
        const double v = std::floor(cum * 4294967296.0);
        a.thr[i] = v >= 4294967296.0 ? 4294967296ull : (uint64_t)v;
    }
    if (cum > 1.0 + 1e-6) return GP_ERR_ARG;
    if (!(q.p_point_replace >= 0.0f && q.p_point_replace <= 1.0f)) return GP_ERR_ARG;
    const double vr = std::floor((double)q.p_point_replace * 4294967296.0);
    a.thr_replace = vr >= 4294967296.0 ? 4294967296ull : (uint64_t)vr;
    if (q.subtree_depth < 0 || q.subtree_depth > 6) return GP_ERR_ARG;
    const uint32_t allowed = ((1u << (GP_MIN + 1)) - 1u) & ~((1u << GP_ADD) - 1u);
    if (q.functions == 0 || (q.functions & ~allowed)) return GP_ERR_ARG;
    for (int op = GP_ADD; op <= GP_MIN; ++op) {
        if (!(q.functions >> op & 1u)) continue;
        a.funcs[a.n_funcs++] = (int16_t)op;
        if (op <= GP_DIV || op >= GP_MAX) a.binary[a.n_binary++] = (int16_t)op;
        else a.unary[a.n_unary++] = (int16_t)op;
    }
    DevCtx *c = nullptr;
    int rc = ctx_of_current(&c);
    if (rc) return rc;
    const size_t need = gp_mutate_workspace_size(n_out);
    void *base = ws;
    if (ws) {
        if (ws_bytes < need || ((uintptr_t)ws & 255u)) return GP_ERR_WORKSPACE;
    } else {
        std::lock_guard<std::mutex> g(g_mu);
        if ((rc = grow(&c->ws, &c->ws_bytes, need))) return rc;
        base = c->ws;
    }
    char *b = static_cast<char *>(base);
    a.progs = progs;
    a.offsets = offsets;
    a.n_progs = n_progs;
    a.n_feat = n_feat;
    a.parents = parents;
    a.n_out = n_out;
    a.subtree_depth = q.subtree_depth;
    a.seed = seed;
    a.offset = offset;
    a.scratch = reinterpret_cast<gp_node *>(b);
    a.lens = reinterpret_cast<int32_t *>(
        b + round_up((int64_t)n_out * 256 * (int64_t)sizeof(gp_node), 256));
    a.kind = out_kind;
    a.out = out_progs;
    a.out_offsets = out_offsets;
    a.dev_status = c->status;
    GP_CUDA(launch_mutate(a, S(stream)));
    return GP_OK;
}

int gp_get_consts(const gp_node *progs, const int32_t *offsets, int n_progs, float *out_consts,
                  void *stream) {
    if (!progs || !offsets || !out_consts || n_progs < 1) return GP_ERR_ARG;
    GP_CUDA(launch_consts(const_cast<gp_node *>(progs), offsets, n_progs, out_consts, false,
                          S(stream)));
    return GP_OK;
}

int gp_set_consts(gp_node *progs, const int32_t *offsets, int n_progs, const float *consts,
                  void *stream) {
    if (!progs || !offsets || !consts || n_progs < 1) return GP_ERR_ARG;
    GP_CUDA(launch_consts(progs, offsets, n_progs, const_cast<float *>(consts), true, S(stream)));
    return GP_OK;
}

int gp_last_device_status(void *stream, uint32_t *flags) {
    if (!flags) return GP_ERR_ARG;
    DevCtx *c = nullptr;
    int rc = ctx_of_current(&c);
    if (rc) return rc;
    GP_CUDA(cudaStreamSynchronize(S(stream)));
    unsigned int v = 0;
    GP_CUDA(cudaMemcpy(&v, c->status, sizeof(v), cudaMemcpyDeviceToHost));
    GP_CUDA(cudaMemset(c->status, 0, sizeof(v)));
    *flags = v;
    return GP_OK;
}

int gp_autotune(const gp_node *progs, const int32_t *offsets, int n_progs, const float *X,
                int64_t n_rows, int n_feat, const float *y, const float *w, int metric,
                gp_eval_opts *best, void *stream) {
    int rc = check_common(progs, offsets, n_progs, X, n_rows, n_feat);
    if (rc) return rc;
    if (!y) return GP_ERR_ARG;
    if ((rc = check_fused_metric(metric))) return rc;
    DevCtx *c = nullptr;
    if ((rc = ctx_of_current(&c))) return rc;
    cudaStream_t st = S(stream);
    // candidates are timed on the first rows only (the column stride stays
    // n_rows): enough work items for the queue to balance, a short search
    const int64_t n_tune = std::min<int64_t>(n_rows, (int64_t)1 << 21);
    float *out = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    GP_CUDA(cudaMalloc(&out, (size_t)n_progs * sizeof(float)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one evaluation with explicit opts on the tuning rows
    auto run = [&](const gp_eval_opts &o) -> int {
        Plan pl;
        int r = make_plan(&o, n_progs, n_tune, n_feat, c, &pl, metric == GP_PEARSON);
        if (r) return r;
        if (pl.L.total > ws_bytes) {
            if (ws) cudaFree(ws);
            ws = nullptr;
            if (cudaMalloc(&ws, pl.L.total) != cudaSuccess) {
                cudaGetLastError();
                ws_bytes = 0;
                return GP_ERR_NOMEM;
            }
            ws_bytes = pl.L.total;
        }
        Workspace W = carve(ws, pl.L, false);
        return run_evaluate(progs, offsets, n_progs, X, n_tune, n_feat, y, w, metric, pl, W, c,
                            out, nullptr, nullptr, st, n_rows);
    };
    // median of three timed calls after one warm-up; +inf if a call fails
    auto time_of = [&](const gp_eval_opts &o, int *err) -> float {
        if ((*err = run(o))) return 3.4e38f;
        float t[3];
        for (int k = 0; k < 3; ++k) {
            cudaEventRecord(e0, st);
            if ((*err = run(o))) return 3.4e38f;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                *err = GP_ERR_CUDA;
                return 3.4e38f;
            }
            cudaEventElapsedTime(&t[k], e0, e1);
        }
        std::sort(t, t + 3);
        return t[1];
    };
    const int fmode = (n_feat <= 2) ? 2 : 0;
    const int64_t base_chunk = default_chunk(n_progs, n_tune, n_feat, c->sms);
    gp_eval_opts best_o{};
    best_o.long_edge = -1;
    float best_ms = 3.4e38f;
    int err = GP_OK;
    // a candidate replaces the best when it is faster by the factor keep
    auto consider = [&](const gp_eval_opts &o, float keep = 1.0f) {
        if (err) return;
        const float ms = time_of(o, &err);
        if (!err && ms < best_ms * keep) {
            best_ms = ms;
            best_o = o;
        }
    };
    // stage 1: rows per thread x chunk length (the default, a half, a
    // quarter: on the 4M x 50 table at 8 rows, 8K-row chunks beat 16K and
    // 4K by 2% and 1%), as many blocks as fit
    for (int rpt : {4, 8})
        for (int64_t ch : {base_chunk, std::max<int64_t>(base_chunk / 2, 1024),
                           std::max<int64_t>(base_chunk / 4, 1024)}) {
            gp_eval_opts o{};
            o.rows_per_thread = rpt;
            o.chunk_rows = (int)round_up(std::min<int64_t>(ch, 65536), 256);
            o.long_edge = -1;
            consider(o);
        }
    // stage 2: fewer resident blocks
    if (!err) {
        const gp_eval_opts b1 = best_o;
        const int occ = eval_info(b1.rows_per_thread, fmode, 0, kEvalBlockThreads, nullptr);
        for (int bps = 1; bps < occ; ++bps) {
            gp_eval_opts o = b1;
            o.blocks_per_sm = bps;
            consider(o);
        }
    }
    // stage 3: a length-bucket edge, the long bucket with its own rows per
    // thread; a split reads the inputs once more and adds a launch, so it
    // must win by 1% (on Pagie-1 16M x 4096 the best split came within
    // 0.3% of one launch, inside the spread of the timings)
    if (!err) {
        const gp_eval_opts b2 = best_o;
        for (int edge : {12, 16, 24, 32})
            for (int lrpt : {4, 8}) {
                gp_eval_opts o = b2;
                o.long_edge = edge;
                o.long_rows_per_thread = lrpt;
                o.long_blocks_per_sm = 0;
                consider(o, 0.99f);
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (ws) cudaFree(ws);
    if (err) return err;
    if (best_o.long_rows_per_thread == 0) best_o.long_rows_per_thread = best_o.rows_per_thread;
    {
        std::lock_guard<std::mutex> g(g_mu);
        c->tuned[ShapeKey{n_progs, n_rows, n_feat}] = best_o;
    }
    if (best) *best = best_o;
    return GP_OK;
}

int gp_probe_pipes(double *out, void *stream) {
    if (!out) return GP_ERR_ARG;
    GP_CUDA(probe_pipes(out, S(stream)));
    return GP_OK;
}

int gp_timing_enable(int on) {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> drop;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_timing.on = on != 0;
        drop.swap(g_timing.live);
    }
    for (auto &e : drop) cudaEventSynchronize(e.second);
    std::lock_guard<std::mutex> g(g_mu);
    for (auto &e : drop) g_timing.pool.push_back(e);
    return GP_OK;
}

int gp_timing_read(double *total_ms, int *n_calls) {
    if (!total_ms) return GP_ERR_ARG;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> live;
    {
        std::lock_guard<std::mutex> g(g_mu);
        live.swap(g_timing.live);
    }
    double sum = 0.0;
    int rc = GP_OK;
    for (auto &e : live) {
        float ms = 0.0f;
        if (cudaEventSynchronize(e.second) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e.first, e.second) != cudaSuccess) {
            cudaGetLastError();
            rc = GP_ERR_CUDA;
        }
        sum += ms;
    }
    {
        std::lock_guard<std::mutex> g(g_mu);
        for (auto &e : live) g_timing.pool.push_back(e);
    }
    *total_ms = sum;
    if (n_calls) *n_calls = (int)live.size();
    return rc;
}

void gp_shutdown(void) {
    std::lock_guard<std::mutex> g(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < kMaxDevices; ++d) {
        DevCtx &c = g_ctx[d];
        if (!c.init) continue;
        cudaSetDevice(d);
        if (c.ws) cudaFree(c.ws);
        if (c.stage) cudaFree(c.stage);
        if (c.rank) cudaFree(c.rank);
        c.ws = c.stage = c.rank = nullptr;
        c.ws_bytes = c.stage_bytes = c.rank_bytes = 0;
        c.tuned.clear();
    }
    cudaSetDevice(cur);
    static_scratch_forget();
}

}  // extern "C"
