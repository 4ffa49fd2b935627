// gp_predict.cu -- the evaluator's interpreter with a store epilogue
// (predictions instead of fitness): gp_predict and the predictions that the
// rank fitness sorts.  One instance per program class, feature columns
// loaded per reference (gp_predict_f2.cu: two columns in registers).
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_predict(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.cls == kClassShallow)
        return launch_eval_t<4, kShallowDepth - 1, 0, kEpiPred, false>(a, grid, block, st);
    if (a.cls == kClassShallow8)
        return launch_eval_t<4, kSmallDepth - 1, 0, kEpiPred, false>(a, grid, block, st);
    if (a.cls == kClassShallowExt)
        return launch_eval_t<4, kSmallDepth - 1, 0, kEpiPred, true>(a, grid, block, st);
    return launch_eval_t<4, kDeepSlots, 0, kEpiPred, true>(a, grid, block, st);
}
int info_predict(int cls, int block, int *regs) {
    if (cls == kClassShallow) return info_t<4, kShallowDepth - 1, 0, kEpiPred, false>(block, regs);
    if (cls == kClassShallow8) return info_t<4, kSmallDepth - 1, 0, kEpiPred, false>(block, regs);
    if (cls == kClassShallowExt) return info_t<4, kSmallDepth - 1, 0, kEpiPred, true>(block, regs);
    return info_t<4, kDeepSlots, 0, kEpiPred, true>(block, regs);
}
}  // namespace gpk
