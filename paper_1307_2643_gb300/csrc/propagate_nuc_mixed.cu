// propagate_nuc_mixed.cu -- the mixed-precision propagate kernels with the
// decay of unstable nuclei held as a third free path in the lane (launched
// when a nuclide table is in use), for the grid field alone and with the
// analytic galactic fields; launch variant 256 x 2 only.  The other mixed
// kernels do not carry the third free path, so their registers are
// unchanged.
#include "propagate_mixed_impl.cuh"

namespace crp {

cudaError_t launch_propagate_mixed_nuc(const KParams& kp, const DevState& st, DevCounters* dc,
                                       int grid, int block, cudaStream_t s) {
  if (kp.flags & CRP_GMF) return launch_policy<PolicyMixedGmfNuc, 256, 2>(kp, st, dc, grid, block, s);
  if (kp.flags & CRP_GALACTIC)
    return launch_policy<PolicyMixedGalNuc, 256, 2>(kp, st, dc, grid, block, s);
  return launch_policy<PolicyMixedNuc, 256, 2>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_mixed_nuc(int dtype, uint32_t flags, int block, int* bps) {
  if (flags & CRP_GMF) return occupancy_policy<PolicyMixedGmfNuc, 256, 2>(dtype, block, bps);
  if (flags & CRP_GALACTIC) return occupancy_policy<PolicyMixedGalNuc, 256, 2>(dtype, block, bps);
  return occupancy_policy<PolicyMixedNuc, 256, 2>(dtype, block, bps);
}

}  // namespace crp
