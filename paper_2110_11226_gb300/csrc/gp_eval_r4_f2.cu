// gp_eval_r4_f2.cu -- instances of the batched evaluator: 4 rows per
// thread, feature mode 2 (columns 0 and 1 held in registers),
// both depth classes (7 or 19 shared-memory stack slots), with the
// loss epilogue or the moment epilogue of the correlation fitness.
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_eval_r4_f2(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.mom) {
        if (a.cls == 0) return launch_eval_t<4, kSmallDepth - 1, 2, kEpiMom>(a, grid, block, st);
        return launch_eval_t<4, kDeepSlots, 2, kEpiMom>(a, grid, block, st);
    }
    if (a.cls == 0) return launch_eval_t<4, kSmallDepth - 1, 2, kEpiLoss>(a, grid, block, st);
    return launch_eval_t<4, kDeepSlots, 2, kEpiLoss>(a, grid, block, st);
}
int info_eval_r4_f2(int cls, int block, int *regs, bool moments) {
    if (moments) {
        if (cls == 0) return info_t<4, kSmallDepth - 1, 2, kEpiMom>(block, regs);
        return info_t<4, kDeepSlots, 2, kEpiMom>(block, regs);
    }
    if (cls == 0) return info_t<4, kSmallDepth - 1, 2, kEpiLoss>(block, regs);
    return info_t<4, kDeepSlots, 2, kEpiLoss>(block, regs);
}
}  // namespace gpk
