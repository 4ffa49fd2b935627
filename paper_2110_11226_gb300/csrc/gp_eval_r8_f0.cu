// gp_eval_r8_f0.cu -- instances of the batched evaluator: 8 rows per
// thread, feature mode 0 (feature columns loaded per reference),
// program class 0 only (6 stack slots; the other classes always run 4 rows
// per thread), with
// the loss epilogue, the moment epilogue of the correlation fitness, or the
// store epilogue (predictions).
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_eval_r8_f0(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.cls != kClassShallow) return cudaErrorInvalidValue;
    if (a.pred) return launch_eval_t<8, kShallowDepth - 1, 0, kEpiPred, false>(a, grid, block, st);
    if (a.mom) return launch_eval_t<8, kShallowDepth - 1, 0, kEpiMom, false>(a, grid, block, st);
    return launch_eval_t<8, kShallowDepth - 1, 0, kEpiLoss, false>(a, grid, block, st);
}
int info_eval_r8_f0(int cls, int block, int *regs, bool moments, bool pred) {
    if (cls != kClassShallow) return 0;
    if (pred) return info_t<8, kShallowDepth - 1, 0, kEpiPred, false>(block, regs);
    if (moments) return info_t<8, kShallowDepth - 1, 0, kEpiMom, false>(block, regs);
    return info_t<8, kShallowDepth - 1, 0, kEpiLoss, false>(block, regs);
}
}  // namespace gpk
