// gp_eval_r16_f0.cu -- instance of the batched evaluator: 16 rows per thread
// in blocks of 4 warps, feature mode 0 (feature columns loaded per reference),
// program class 0 only (6 stack slots; the other classes always run 4 rows
// per thread).
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_eval_r16_f0(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.cls != kClassShallow || a.mom) return cudaErrorInvalidValue;
    return launch_eval_t<16, kShallowDepth - 1, 0, kEpiLoss, false>(a, grid, block, st);
}
int info_eval_r16_f0(int cls, int block, int *regs, bool moments) {
    if (cls != kClassShallow || moments) return 0;
    return info_t<16, kShallowDepth - 1, 0, kEpiLoss, false>(block, regs);
}
}  // namespace gpk
