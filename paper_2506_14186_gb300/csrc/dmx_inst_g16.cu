// Kernel instantiation for 16 lane(s) per environment (one translation unit
// per lane count so that the build compiles them in parallel).
#include "dmx_kernels.cuh"

namespace dmx {
template cudaError_t launch_persistent_g<16>(const RolloutParams&, int, int, size_t, cudaStream_t);
template cudaError_t launch_step_g<16>(const RolloutParams&, const StepState&, bool, int, size_t, cudaStream_t);
template int occupancy_g<16>(int, size_t);
template cudaError_t launch_eval_rhs_g<16>(const RolloutParams&, const double*, const double*, const double*, int,
                                            double*, int*, int, size_t, cudaStream_t);
}  // namespace dmx
