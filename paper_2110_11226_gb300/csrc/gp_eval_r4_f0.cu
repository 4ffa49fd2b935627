// gp_eval_r4_f0.cu -- instances of the batched evaluator: 4 rows per
// thread, feature mode 0 (feature columns loaded per reference),
// both depth classes (7 or 19 shared-memory stack slots), with the
// loss epilogue or the moment epilogue of the correlation fitness.
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_eval_r4_f0(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.mom) {
        if (a.cls == 0) return launch_eval_t<4, kSmallDepth - 1, 0, kEpiMom>(a, grid, block, st);
        return launch_eval_t<4, kDeepSlots, 0, kEpiMom>(a, grid, block, st);
    }
    if (a.cls == 0) return launch_eval_t<4, kSmallDepth - 1, 0, kEpiLoss>(a, grid, block, st);
    return launch_eval_t<4, kDeepSlots, 0, kEpiLoss>(a, grid, block, st);
}
int info_eval_r4_f0(int cls, int block, int *regs, bool moments) {
    if (moments) {
        if (cls == 0) return info_t<4, kSmallDepth - 1, 0, kEpiMom>(block, regs);
        return info_t<4, kDeepSlots, 0, kEpiMom>(block, regs);
    }
    if (cls == 0) return info_t<4, kSmallDepth - 1, 0, kEpiLoss>(block, regs);
    return info_t<4, kDeepSlots, 0, kEpiLoss>(block, regs);
}
}  // namespace gpk
