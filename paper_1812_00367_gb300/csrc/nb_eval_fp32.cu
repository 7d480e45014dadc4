// nb_eval_fp32.cu -- FP32 instantiations of the evaluation kernel (nb_eval.cuh).
#include "nb_eval.cuh"

namespace nb {

cudaError_t launch_eval_fp32(const Dev &d, int mode, const EvalLaunch &L, int grid,
                             cudaStream_t st) {
    switch (mode) {
    case kModeOut: return launch_eval_t<NB_FP32, kModeOut>(d, L, grid, st);
    case kModeStep: return launch_eval_t<NB_FP32, kModeStep>(d, L, grid, st);
    case kModeInit1: return launch_eval_t<NB_FP32, kModeInit1>(d, L, grid, st);
    case kModeInit2: return launch_eval_t<NB_FP32, kModeInit2>(d, L, grid, st);
    case kModeOut4: return launch_eval_t<NB_FP32, kModeOut4>(d, L, grid, st);
    case kModeStep4: return launch_eval_t<NB_FP32, kModeStep4>(d, L, grid, st);
    case kModeInit4: return launch_eval_t<NB_FP32, kModeInit4>(d, L, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

int occupancy_fp32(int mode) {
    if (is_order4_mode(mode)) return occupancy_t<NB_FP32, kModeStep4>();
    return occupancy_t<NB_FP32, kModeStep>();
}

}  // namespace nb
