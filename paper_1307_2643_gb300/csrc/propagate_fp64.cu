// propagate_fp64.cu -- binary64 propagate kernels.  Built with -fmad=false:
// every multiply and add is rounded separately, in source order.
#include "propagate.cuh"

namespace crp {

cudaError_t launch_propagate_fp64(const KParams& kp, const DevState& st, DevCounters* dc,
                                  int grid, int block, cudaStream_t s) {
  return launch_policy<PolicyFP64, 2>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_fp64(int dtype, int block, int* bps) {
  return occupancy_policy<PolicyFP64, 2>(dtype, block, bps);
}

size_t propagate_smem_fp64(int block) { return smem_bytes<PolicyFP64>(block); }

}  // namespace crp
