// propagate_mixed.cu -- mixed-precision propagate kernels (binary32 field,
// force and Runge-Kutta stages; binary64 positions, lengths, energies, free
// paths and error norm).  The multi-arm galactic policy is instantiated in
// propagate_gmf.cu, the fixed extragalactic module list in propagate_egal.cu.
#include "propagate_mixed_impl.cuh"

namespace crp {

cudaError_t launch_propagate_mixed(const KParams& kp, const DevState& st, DevCounters* dc,
                                   int grid, int block, int variant, cudaStream_t s) {
  if (kp.flags & CRP_GMF) return launch_propagate_mixed_gmf(kp, st, dc, grid, block, variant, s);
  if (kp.flags == kEgalModules && variant == 2)
    return launch_propagate_mixed_egal(kp, st, dc, grid, block, s);
  return (kp.flags & CRP_GALACTIC)
             ? launch_variant<PolicyMixedGal>(kp, st, dc, grid, block, variant, s)
             : launch_variant<PolicyMixed>(kp, st, dc, grid, block, variant, s);
}

// galactic: 0 none, 1 analytic disk + halo, 2 multi-arm field (with or without
// it), 3 the fixed extragalactic module list (variant 2)
cudaError_t occupancy_propagate_mixed(int dtype, int galactic, int variant, int block, int* bps) {
  if (galactic == 2) return occupancy_propagate_mixed_gmf(dtype, variant, block, bps);
  if (galactic == 3 && variant == 2) return occupancy_propagate_mixed_egal(dtype, block, bps);
  return galactic ? occupancy_variant<PolicyMixedGal>(dtype, variant, block, bps)
                  : occupancy_variant<PolicyMixed>(dtype, variant, block, bps);
}

size_t propagate_smem_mixed(int block) { return smem_bytes<PolicyMixed>(block); }

cudaError_t sample_field_mixed(const KParams& kp, const double* xyz, int64_t n, double* B,
                               cudaStream_t s) {
  if (kp.flags & CRP_GMF) return sample_field_mixed_gmf(kp, xyz, n, B, s);
  return (kp.flags & CRP_GALACTIC) ? sample_policy<PolicyMixedGal>(kp, xyz, n, B, s)
                                   : sample_policy<PolicyMixed>(kp, xyz, n, B, s);
}

}  // namespace crp
