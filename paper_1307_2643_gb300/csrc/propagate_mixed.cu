// propagate_mixed.cu -- mixed-precision propagate kernels (binary32 field,
// force and Runge-Kutta stages; binary64 positions, lengths, energies, free
// paths and error norm).
#include "propagate.cuh"

namespace crp {

cudaError_t launch_propagate_mixed(const KParams& kp, const DevState& st, DevCounters* dc,
                                   int grid, int block, cudaStream_t s) {
  return launch_policy<PolicyMixed>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_mixed(int dtype, int block, int* bps) {
  return occupancy_policy<PolicyMixed>(dtype, block, bps);
}

size_t propagate_smem_mixed(int block) { return smem_bytes<PolicyMixed>(block); }

}  // namespace crp
