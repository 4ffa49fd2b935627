// gp_eval_r4_f0.cu -- instances of the batched evaluator: 4 rows per
// thread, feature mode 0 (feature columns loaded per reference),
// all four program classes (6 shared-memory stack slots for class 0, 7 for
// class 3 and for class 2 with the extended functions, 19 slots with every
// function), with the loss epilogue or the moment epilogue of the
// correlation fitness.
#include "gp_interp.cuh"

namespace gpk {
namespace {
template <int EPI>
cudaError_t launch_cls(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    if (a.cls == kClassShallow)
        return launch_eval_t<4, kShallowDepth - 1, 0, EPI, false>(a, grid, block, st);
    if (a.cls == kClassShallow8)
        return launch_eval_t<4, kSmallDepth - 1, 0, EPI, false>(a, grid, block, st);
    if (a.cls == kClassShallowExt)
        return launch_eval_t<4, kSmallDepth - 1, 0, EPI, true>(a, grid, block, st);
    return launch_eval_t<4, kDeepSlots, 0, EPI, true>(a, grid, block, st);
}
template <int EPI>
int info_cls(int cls, int block, int *regs) {
    if (cls == kClassShallow) return info_t<4, kShallowDepth - 1, 0, EPI, false>(block, regs);
    if (cls == kClassShallow8) return info_t<4, kSmallDepth - 1, 0, EPI, false>(block, regs);
    if (cls == kClassShallowExt) return info_t<4, kSmallDepth - 1, 0, EPI, true>(block, regs);
    return info_t<4, kDeepSlots, 0, EPI, true>(block, regs);
}
}  // namespace

cudaError_t launch_eval_r4_f0(const EvalArgs &a, int grid, int block, cudaStream_t st) {
    return a.mom ? launch_cls<kEpiMom>(a, grid, block, st) : launch_cls<kEpiLoss>(a, grid, block, st);
}
int info_eval_r4_f0(int cls, int block, int *regs, bool moments) {
    return moments ? info_cls<kEpiMom>(cls, block, regs) : info_cls<kEpiLoss>(cls, block, regs);
}
}  // namespace gpk
