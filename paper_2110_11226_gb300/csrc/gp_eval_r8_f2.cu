// gp_eval_r8_f2.cu -- instances of the batched evaluator: 8 rows per
// thread, feature mode 2 (columns 0 and 1 held in registers),
// both depth classes (7 or 19 shared-memory stack slots).
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_eval_r8_f2(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.cls == 0) return launch_eval_t<8, kSmallDepth - 1, 2, false>(a, grid, block, st);
    return launch_eval_t<8, kDeepSlots, 2, false>(a, grid, block, st);
}
int info_eval_r8_f2(int cls, int block, int *regs) {
    if (cls == 0) return info_t<8, kSmallDepth - 1, 2, false>(block, regs);
    return info_t<8, kDeepSlots, 2, false>(block, regs);
}
}  // namespace gpk
