// gp_reduce.cu -- cross-block fitness reduction (the weighted column sum of
// Sec. III-C3): one warp per program adds that program's per-chunk partial
// sums in a fixed order, in FP64 (default) or Kahan-compensated FP32, and
// divides by the total weight.
#include "gp_internal.cuh"

namespace gpk {

__device__ __forceinline__ void kahan32(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = isfinite(t) ? __fsub_rn(__fsub_rn(t, s), y) : 0.0f;
    s = t;
}

__device__ __forceinline__ double finish_metric(int metric, double s_e, double s_w) {
    double f = s_e / s_w;
    if (metric == GP_RMSE) f = sqrt(f);
    return f;
}

// |r| of the weighted Pearson correlation from shifted moment sums:
// s1 = sum w d, s2 = sum w d^2, s12 = sum w d yc (d = p - shift), with
// syc = sum w yc, syy = sum w yc^2 and sw = sum w.  Shifting p or y by a
// constant leaves r unchanged.  Non-finite sums give NaN; a zero variance
// gives 0.
__device__ double pearson_from_moments(double s1, double s2, double s12, double sw, double syc,
                                       double syy) {
    const double md = s1 / sw, my = syc / sw;
    const double vp = s2 / sw - md * md;
    const double vy = syy / sw - my * my;
    const double cov = s12 / sw - md * my;
    if (!isfinite(vp) || !isfinite(cov) || !isfinite(vy))
        return __longlong_as_double(0x7ff8000000000000LL);
    if (!(vp > 0.0) || !(vy > 0.0)) return 0.0;
    return fabs(cov) / sqrt(vp * vy);
}

// warp w handles program w; lane l adds chunks l, l+32, ... in order, then
// the 32 lane sums are combined by lane 0 in lane order.
__global__ void __launch_bounds__(256) finalize_kernel(FinalizeArgs a) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (p >= a.n_progs) return;
    const float *part = a.part + (size_t)p * a.n_chunks;
    const ProgMeta m = a.meta[p];
    double f;
    if (a.mom) {
        // correlation fitness: the moment sums of d = p - shift and yc,
        // chunk order per lane then lane order, in FP64
        const double *mp = a.mom + (size_t)p * a.n_chunks * 3;
        double s[3] = {0.0, 0.0, 0.0};
        for (int i = lane; i < a.n_chunks; i += 32)
            for (int k = 0; k < 3; ++k) s[k] += mp[(size_t)i * 3 + k];
        double S[3] = {0.0, 0.0, 0.0};
        for (int l = 0; l < 32; ++l)
            for (int k = 0; k < 3; ++k) S[k] += __shfl_sync(0xffffffffu, s[k], l);
        f = pearson_from_moments(S[0], S[1], S[2], *a.sumw, a.ystat[1], a.ystat[2]);
    } else if (a.accum == GP_ACCUM_KAHAN32) {
        float s = 0.0f, c = 0.0f;
        for (int i = lane; i < a.n_chunks; i += 32) kahan32(s, c, part[i]);
        float mine = __fsub_rn(s, c);
        float S = 0.0f, Cc = 0.0f;
        for (int l = 0; l < 32; ++l) {
            const float v = __shfl_sync(0xffffffffu, mine, l);
            kahan32(S, Cc, v);
        }
        f = finish_metric(a.metric, (double)__fsub_rn(S, Cc), *a.sumw);
        f = (double)(float)f;
    } else {
        double s = 0.0;
        for (int i = lane; i < a.n_chunks; i += 32) s += (double)part[i];
        double S = 0.0;
        for (int l = 0; l < 32; ++l) S += __shfl_sync(0xffffffffu, s, l);
        f = finish_metric(a.metric, S, *a.sumw);
    }
    if (m.status != GP_PROG_OK) f = __longlong_as_double(0x7ff8000000000000LL);
    if (lane == 0) {
        a.out[p] = (float)f;
        if (a.out64) a.out64[p] = f;
        if (a.out_prog_status) a.out_prog_status[p] = m.status;
    }
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t st) {
    if (a.n_progs <= 0) return cudaSuccess;
    const int warps = 8;
    const int grid = (a.n_progs + warps - 1) / warps;
    finalize_kernel<<<grid, warps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

// constant gradients: same order; grad = S_g / S_w, RMSE scaled by 1/(2 RMSE)
__global__ void __launch_bounds__(256) grad_finalize_kernel(GradFinalizeArgs a) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (p >= a.n_progs) return;
    const ProgMeta m = a.meta[p];
    const double sw = *a.sumw;
    double s = 0.0;
    for (int i = lane; i < a.n_chunks; i += 32) s += (double)a.part[(size_t)p * a.n_chunks + i];
    double S = 0.0;
    for (int l = 0; l < 32; ++l) S += __shfl_sync(0xffffffffu, s, l);
    double f = finish_metric(a.metric, S, sw);
    const bool bad = (m.status != GP_PROG_OK) || (m.n_consts > GP_MAX_CONSTS);
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    double scale = 1.0 / sw;
    if (a.metric == GP_RMSE) scale = (f > 0.0) ? scale / (2.0 * f) : 0.0;
    // lanes 0..15 each finish one constant slot
    double g = 0.0;
    if (lane < GP_MAX_CONSTS) {
        const float *gp = a.gpart + (size_t)p * a.n_chunks * GP_MAX_CONSTS + lane;
        for (int i = 0; i < a.n_chunks; ++i) g += (double)gp[(size_t)i * GP_MAX_CONSTS];
        g = (lane < m.n_consts) ? g * scale : 0.0;
        if (bad) g = nan;
        a.grad[(size_t)p * GP_MAX_CONSTS + lane] = (float)g;
    }
    if (lane == 0 && a.fit) a.fit[p] = (float)(m.status != GP_PROG_OK ? nan : f);
}

cudaError_t launch_grad_finalize(const GradFinalizeArgs &a, cudaStream_t st) {
    if (a.n_progs <= 0) return cudaSuccess;
    const int warps = 8;
    const int grid = (a.n_progs + warps - 1) / warps;
    grad_finalize_kernel<<<grid, warps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gpk
