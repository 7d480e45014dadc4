// nb_eval_ex.cu -- EX instantiations of the evaluation kernel (nb_eval.cuh).
#include "nb_eval.cuh"

namespace nb {

cudaError_t launch_eval_ex(const Dev &d, int mode, const EvalLaunch &L, int grid,
                             cudaStream_t st) {
    switch (mode) {
    case kModeOut: return launch_eval_t<NB_EX, kModeOut>(d, L, grid, st);
    case kModeStep: return launch_eval_t<NB_EX, kModeStep>(d, L, grid, st);
    case kModeInit1: return launch_eval_t<NB_EX, kModeInit1>(d, L, grid, st);
    case kModeInit2: return launch_eval_t<NB_EX, kModeInit2>(d, L, grid, st);
    case kModeOut4: return launch_eval_t<NB_EX, kModeOut4>(d, L, grid, st);
    case kModeStep4: return launch_eval_t<NB_EX, kModeStep4>(d, L, grid, st);
    case kModeInit4: return launch_eval_t<NB_EX, kModeInit4>(d, L, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

int occupancy_ex(int mode) {
    if (is_order4_mode(mode)) return occupancy_t<NB_EX, kModeStep4>();
    return occupancy_t<NB_EX, kModeStep>();
}

}  // namespace nb
