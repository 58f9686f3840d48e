// Multi-stage (Runge-Kutta) forms on the generic kernels: fused steps on the
// trapezoid tiles and combining stages on the direct kernel or the column
// march.  Its own translation unit, so that these instances build in parallel
// with the rest.
#include "generic_kernels.cuh"

namespace lope {

cudaError_t launch_generic_rk(const StepArgs& a, int kind, int* blocks) {
  return dispatch_generic<true>(a, kind, blocks);
}

}  // namespace lope
