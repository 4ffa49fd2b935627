// gp_static.cu -- gp_evaluate_static: the batched evaluator driven with a
// scratch area that is part of the library's own device image instead of
// memory allocated at run time.
//
// Some callers cannot allocate device memory when they evaluate: a serving
// process whose device memory is all handed out at start-up to another
// allocator, code that must not call cudaMalloc/cudaFree because those can
// synchronise the whole device, or a caller that owns no allocator at all.
// They get this entry point: it uses a fixed, file-scope __device__ array as
// the evaluator's workspace, so it performs no allocation of any kind.
#include <mutex>

#include "gp_internal.cuh"

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_gp_static_scratch[GP_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxStaticDevices];  // device address of the array, per device

// The array's name is only a host-side handle; its device address is looked
// up once per device, with that device current.
int static_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxStaticDevices) {
        cudaGetLastError();
        return GP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gp_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GP_ERR_CUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return GP_OK;
}

}  // namespace

namespace gpk {
// the device addresses are good for the life of each device's context;
// gp_shutdown forgets them (a later call looks them up again)
void static_scratch_forget() {
    std::lock_guard<std::mutex> g(g_static_mu);
    for (int d = 0; d < kMaxStaticDevices; ++d) g_static_ptr[d] = nullptr;
}
}  // namespace gpk

// The default tunables, or, when their workspace does not fit the array,
// longer row chunks (fewer per-chunk partial sums): 65536 rows, then 4x
// longer each time.  opts->chunk_rows = 0 means the defaults.
extern "C" int gp_static_opts(int n_progs, int64_t n_rows, int n_feat, int metric,
                              gp_eval_opts *out) {
    if (n_progs < 1 || n_rows < 1 || n_feat < 1 || !out) return GP_ERR_ARG;
    gp_eval_opts opts{};
    size_t need = gpk::workspace_bytes_for(n_progs, n_rows, n_feat, nullptr, metric);
    if (need == 0) return GP_ERR_ARG;
    for (int chunk = 65536; need > (size_t)GP_STATIC_SCRATCH_BYTES && chunk <= (1 << 22);
         chunk *= 4) {
        opts.chunk_rows = chunk;
        need = gpk::workspace_bytes_for(n_progs, n_rows, n_feat, &opts, metric);
        if (need == 0) return GP_ERR_ARG;
    }
    if (need > (size_t)GP_STATIC_SCRATCH_BYTES) return GP_ERR_WORKSPACE;
    *out = opts;
    return GP_OK;
}

extern "C" int gp_evaluate_static(const gp_node *progs, const int32_t *offsets, int n_progs,
                                  const float *X, int64_t n_rows, int n_feat, const float *y,
                                  const float *w, int metric, float *out_fitness, void *stream) {
    gp_eval_opts opts{};
    int rc = gp_static_opts(n_progs, n_rows, n_feat, metric, &opts);
    if (rc != GP_OK) return rc;
    void *ws = nullptr;
    rc = static_scratch(&ws);
    if (rc != GP_OK) return rc;
    // the evaluator clears the one region that must start at zero (the work
    // queue counters) on every call and writes every other region before
    // reading it, so nothing of the previous call leaks into this one
    return gp_evaluate_ex(progs, offsets, n_progs, X, n_rows, n_feat, y, w, metric,
                          opts.chunk_rows ? &opts : nullptr, out_fitness, nullptr, nullptr, ws,
                          (size_t)GP_STATIC_SCRATCH_BYTES, stream);
}
