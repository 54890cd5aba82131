// propagate_egal.cu -- the mixed-precision propagate kernel for the
// extragalactic module list (pair production, adiabatic loss, pion
// production, E_min, observer) fixed at compile time, in a unit of its own.
// Without the run-time flag tests the unused modules' code and registers drop
// out (no spills at 128 registers).  Results equal the generic kernel's.
#include "propagate_mixed_impl.cuh"

namespace crp {

cudaError_t launch_propagate_mixed_egal(const KParams& kp, const DevState& st, DevCounters* dc,
                                        int grid, int block, cudaStream_t s) {
  return launch_policy<PolicyMixedEgal, 256, 2>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_mixed_egal(int dtype, int block, int* bps) {
  return occupancy_policy<PolicyMixedEgal, 256, 2>(dtype, block, bps);
}

}  // namespace crp
