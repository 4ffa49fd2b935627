// gp_select.cu -- tournament selection on the device (Sec. III-C1): one
// thread per tournament, k draws from Philox4x32-10, the best adjusted
// fitness wins (Eqs. parsimony and fitness).
#include <math_constants.h>

#include "gp_internal.cuh"

namespace gpk {

__global__ void __launch_bounds__(256) tournament_kernel(TournArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tourn) return;
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    int best = -1;
    double best_adj = 0.0;
    uint4 r = make_uint4(0, 0, 0, 0);
    for (int j = 0; j < a.k; ++j) {
        if ((j & 3) == 0)
            r = philox4x32_10(make_uint4((uint32_t)(j >> 2), (uint32_t)t, (uint32_t)a.offset,
                                         (uint32_t)(a.offset >> 32)),
                              key);
        const uint32_t u = (j & 3) == 0 ? r.x : (j & 3) == 1 ? r.y : (j & 3) == 2 ? r.z : r.w;
        const int i = (int)(((uint64_t)u * (uint64_t)a.n_progs) >> 32);
        // adjusted fitness in FP64 so the comparison is decided exactly as
        // a double-precision reference decides it
        double pen = 0.0;
        if (a.offsets)
            pen = __dmul_rn((double)a.parsimony, (double)(a.offsets[i + 1] - a.offsets[i]));
        const double raw = (double)a.fitness[i];
        double adj;
        bool better;
        if (a.greater) {
            adj = __dsub_rn(raw, pen);
            if (isnan(adj)) adj = -CUDART_INF;
            better = best < 0 || adj > best_adj;
        } else {
            adj = __dadd_rn(raw, pen);
            if (isnan(adj)) adj = CUDART_INF;
            better = best < 0 || adj < best_adj;
        }
        if (better) {
            best = i;
            best_adj = adj;
        }
    }
    a.out[t] = best;
}

cudaError_t launch_tournament(const TournArgs &a, cudaStream_t st) {
    if (a.n_tourn <= 0) return cudaSuccess;
    const int block = 256;
    tournament_kernel<<<(a.n_tourn + block - 1) / block, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gpk
