// The two-pass update kernels (dense and compact layouts) for the __half storage.
#include "lbm_compact_update.cuh"
#include "lbm_twopass.cuh"

namespace lbm {

template cudaError_t launch_two_pass_t<__half>(const StepArgs &);
template cudaError_t launch_compact_t<__half>(const StepArgs &, int);
template cudaError_t launch_persist_t<__half>(const StepArgs &, int);

}  // namespace lbm
