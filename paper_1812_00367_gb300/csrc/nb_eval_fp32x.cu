// nb_eval_fp32x.cu -- FP32X instantiations of the evaluation kernel
// (nb_eval.cuh): float-float acceleration and potential, FP32 jerk and snap.
#include "nb_eval.cuh"

namespace nb {

cudaError_t launch_eval_fp32x(const Dev &d, int mode, const EvalLaunch &L, int grid,
                              cudaStream_t st) {
    switch (mode) {
    case kModeOut: return launch_eval_t<NB_FP32X, kModeOut>(d, L, grid, st);
    case kModeStep: return launch_eval_t<NB_FP32X, kModeStep>(d, L, grid, st);
    case kModeInit1: return launch_eval_t<NB_FP32X, kModeInit1>(d, L, grid, st);
    case kModeInit2: return launch_eval_t<NB_FP32X, kModeInit2>(d, L, grid, st);
    case kModeOut4: return launch_eval_t<NB_FP32X, kModeOut4>(d, L, grid, st);
    case kModeStep4: return launch_eval_t<NB_FP32X, kModeStep4>(d, L, grid, st);
    case kModeInit4: return launch_eval_t<NB_FP32X, kModeInit4>(d, L, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

int occupancy_fp32x(int mode) {
    if (is_order4_mode(mode)) return occupancy_t<NB_FP32X, kModeStep4>();
    return occupancy_t<NB_FP32X, kModeStep>();
}

}  // namespace nb
