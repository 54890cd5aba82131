// propagate_nuc_fp64.cu -- the binary64 propagate kernel with the decay of
// unstable nuclei held as a third free path in the lane (launched when a
// nuclide table is in use).  Compiled with -fmad=false, like the other
// binary64 kernels, so its arithmetic is the oracle's operation for
// operation.
#include "propagate.cuh"

namespace crp {

cudaError_t launch_propagate_fp64_nuc(const KParams& kp, const DevState& st, DevCounters* dc,
                                      int grid, int block, cudaStream_t s) {
  return launch_policy<PolicyFP64Nuc, 128, 2>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_fp64_nuc(int dtype, int block, int* bps) {
  return occupancy_policy<PolicyFP64Nuc, 128, 2>(dtype, block, bps);
}

}  // namespace crp
