// gp_predict.cu -- the evaluator's interpreter with a store epilogue
// (predictions instead of fitness), for parity checks of single rows.
#include "gp_interp.cuh"

namespace gpk {
cudaError_t launch_predict(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    return launch_eval_t<4, kDeepSlots, 0, kEpiPred>(a, grid, block, st);
}
int info_predict(int block, int *regs) { return info_t<4, kDeepSlots, 0, kEpiPred>(block, regs); }
}  // namespace gpk
