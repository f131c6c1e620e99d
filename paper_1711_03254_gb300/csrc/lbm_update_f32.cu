// The two-pass update kernels (dense and compact layouts) for the float storage.
#include "lbm_compact_update.cuh"
#include "lbm_twopass.cuh"

namespace lbm {

template cudaError_t launch_two_pass_t<float>(const StepArgs &);
template cudaError_t launch_compact_t<float>(const StepArgs &, int);
template cudaError_t launch_persist_t<float>(const StepArgs &, int);

}  // namespace lbm
