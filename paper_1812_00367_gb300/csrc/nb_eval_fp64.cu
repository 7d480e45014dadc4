// nb_eval_fp64.cu -- FP64 instantiations of the evaluation kernel (nb_eval.cuh).
#include "nb_eval.cuh"

namespace nb {

cudaError_t launch_eval_fp64(const Dev &d, int mode, const EvalLaunch &L, int grid,
                             cudaStream_t st) {
    switch (mode) {
    case kModeOut: return launch_eval_t<NB_FP64, kModeOut>(d, L, grid, st);
    case kModeStep: return launch_eval_t<NB_FP64, kModeStep>(d, L, grid, st);
    case kModeInit1: return launch_eval_t<NB_FP64, kModeInit1>(d, L, grid, st);
    case kModeInit2: return launch_eval_t<NB_FP64, kModeInit2>(d, L, grid, st);
    case kModeOut4: return launch_eval_t<NB_FP64, kModeOut4>(d, L, grid, st);
    case kModeStep4: return launch_eval_t<NB_FP64, kModeStep4>(d, L, grid, st);
    case kModeInit4: return launch_eval_t<NB_FP64, kModeInit4>(d, L, grid, st);
    case kModePot: return launch_eval_t<NB_FP64, kModePot>(d, L, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

int occupancy_fp64(int mode) {
    if (mode == kModePot) return occupancy_t<NB_FP64, kModePot>();
    if (is_order4_mode(mode)) return occupancy_t<NB_FP64, kModeStep4>();
    return occupancy_t<NB_FP64, kModeStep>();
}

}  // namespace nb
