// propagate_mixed.cu -- mixed-precision propagate kernels (binary32 field,
// force and Runge-Kutta stages; binary64 positions, lengths, energies, free
// paths and error norm).
#include "propagate.cuh"

namespace crp {

// Register-allocation variants: sized for 2 resident 256-thread blocks per
// SM (no spills) or for 3 (more warps to hide gather latency).
cudaError_t launch_propagate_mixed(const KParams& kp, const DevState& st, DevCounters* dc,
                                   int grid, int block, int variant, cudaStream_t s) {
  const bool gal = (kp.flags & CRP_GALACTIC) != 0;
  if (variant == 3)
    return gal ? launch_policy<PolicyMixedGal, 3>(kp, st, dc, grid, block, s)
               : launch_policy<PolicyMixed, 3>(kp, st, dc, grid, block, s);
  return gal ? launch_policy<PolicyMixedGal, 2>(kp, st, dc, grid, block, s)
             : launch_policy<PolicyMixed, 2>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_mixed(int dtype, int galactic, int variant, int block, int* bps) {
  if (variant == 3)
    return galactic ? occupancy_policy<PolicyMixedGal, 3>(dtype, block, bps)
                    : occupancy_policy<PolicyMixed, 3>(dtype, block, bps);
  return galactic ? occupancy_policy<PolicyMixedGal, 2>(dtype, block, bps)
                  : occupancy_policy<PolicyMixed, 2>(dtype, block, bps);
}

size_t propagate_smem_mixed(int block) { return smem_bytes<PolicyMixed>(block); }

}  // namespace crp
