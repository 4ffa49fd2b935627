// gp_eval_r8_f0.cu -- instances of the batched evaluator: 8 rows per
// thread, feature mode 0 (feature columns loaded per reference),
// both depth classes (7 or 19 shared-memory stack slots);
// the moment epilogue of the correlation fitness for the shallow class (the
// deep class always runs 4 rows per thread).
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_eval_r8_f0(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.mom) {
        if (a.cls != 0) return cudaErrorInvalidValue;
        return launch_eval_t<8, kSmallDepth - 1, 0, kEpiMom>(a, grid, block, st);
    }
    if (a.cls == 0) return launch_eval_t<8, kSmallDepth - 1, 0, kEpiLoss>(a, grid, block, st);
    return launch_eval_t<8, kDeepSlots, 0, kEpiLoss>(a, grid, block, st);
}
int info_eval_r8_f0(int cls, int block, int *regs, bool moments) {
    if (moments) return cls == 0 ? info_t<8, kSmallDepth - 1, 0, kEpiMom>(block, regs) : 0;
    if (cls == 0) return info_t<8, kSmallDepth - 1, 0, kEpiLoss>(block, regs);
    return info_t<8, kDeepSlots, 0, kEpiLoss>(block, regs);
}
}  // namespace gpk
