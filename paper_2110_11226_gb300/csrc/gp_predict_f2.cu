// gp_predict_f2.cu -- the store-epilogue instances (predictions) for tables
// of at most two columns, held in registers (feature mode 2), one per
// program class.
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_predict_f2(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.cls == kClassShallow)
        return launch_eval_t<4, kShallowDepth - 1, 2, kEpiPred, false>(a, grid, block, st);
    if (a.cls == kClassShallow8)
        return launch_eval_t<4, kSmallDepth - 1, 2, kEpiPred, false>(a, grid, block, st);
    if (a.cls == kClassShallowExt)
        return launch_eval_t<4, kSmallDepth - 1, 2, kEpiPred, true>(a, grid, block, st);
    return launch_eval_t<4, kDeepSlots, 2, kEpiPred, true>(a, grid, block, st);
}
int info_predict_f2(int cls, int block, int *regs) {
    if (cls == kClassShallow) return info_t<4, kShallowDepth - 1, 2, kEpiPred, false>(block, regs);
    if (cls == kClassShallow8) return info_t<4, kSmallDepth - 1, 2, kEpiPred, false>(block, regs);
    if (cls == kClassShallowExt) return info_t<4, kSmallDepth - 1, 2, kEpiPred, true>(block, regs);
    return info_t<4, kDeepSlots, 2, kEpiPred, true>(block, regs);
}
}  // namespace gpk
