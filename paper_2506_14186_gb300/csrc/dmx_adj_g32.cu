// Reverse-mode adjoint kernels for 32 lanes per environment (one translation
// unit per lane count so that the build compiles them in parallel).
#include "dmx_adjoint_rev.cuh"

namespace dmx {
template cudaError_t launch_adjoint_rev_g<32>(const AdjParams&, int, int, size_t, cudaStream_t);
template int occupancy_adjoint_rev_g<32>(int, size_t);
template cudaError_t launch_eval_rhs_vjp_g<32>(const AdjParams&, const double*, const double*, const double*,
                                              const double*, double*, double*, double*, int*, int, size_t,
                                              cudaStream_t);
}  // namespace dmx
