// propagate_mixed.cu -- mixed-precision propagate kernels (binary32 field,
// force and Runge-Kutta stages; binary64 positions, lengths, energies, free
// paths and error norm).  The multi-arm galactic policy is instantiated in
// propagate_gmf.cu, the fixed common module lists in propagate_fixed.cu.
#include "propagate_mixed_impl.cuh"

namespace crp {

cudaError_t launch_propagate_mixed(const KParams& kp, const DevState& st, DevCounters* dc,
                                   int grid, int block, int variant, cudaStream_t s) {
  if (kp.nuc_tab) return launch_propagate_mixed_nuc(kp, st, dc, grid, block, s);
  if (variant == 2) {
    const int fx = fixed_modules_index(kp.flags);
    if (fx >= 0) return launch_propagate_mixed_fixed(fx, kp, st, dc, grid, block, s);
  }
  if (kp.flags & CRP_GMF) return launch_propagate_mixed_gmf(kp, st, dc, grid, block, variant, s);
  return (kp.flags & CRP_GALACTIC)
             ? launch_variant<PolicyMixedGal>(kp, st, dc, grid, block, variant, s)
             : launch_variant<PolicyMixed>(kp, st, dc, grid, block, variant, s);
}

// the kernel launch_propagate_mixed would run for these flags and variant
cudaError_t occupancy_propagate_mixed(int dtype, uint32_t flags, int variant, int block, int* bps,
                                      bool nuc) {
  if (nuc) return occupancy_propagate_mixed_nuc(dtype, flags, block, bps);
  if (variant == 2) {
    const int fx = fixed_modules_index(flags);
    if (fx >= 0) return occupancy_propagate_mixed_fixed(fx, dtype, block, bps);
  }
  if (flags & CRP_GMF) return occupancy_propagate_mixed_gmf(dtype, flags, variant, block, bps);
  return (flags & CRP_GALACTIC) ? occupancy_variant<PolicyMixedGal>(dtype, variant, block, bps)
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
