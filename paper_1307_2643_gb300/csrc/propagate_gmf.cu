// propagate_gmf.cu -- the mixed-precision propagate kernels with the analytic
// multi-arm galactic field (CRP_GMF), in a unit of their own: the disk + halo
// and plain policies stay free of its code and registers.
#include "propagate_mixed_impl.cuh"

namespace crp {

namespace {
// back-tracking through the multi-arm field to the galaxy border, with the
// module list fixed at compile time (records byte-identical to the generic
// kernel's)
using PolicyGmfBorder = PolicyMixedT<true, true, kModsGmfBorder>;
}  // namespace

cudaError_t launch_propagate_mixed_gmf(const KParams& kp, const DevState& st, DevCounters* dc,
                                       int grid, int block, int variant, cudaStream_t s) {
  if (variant == 2 && kp.flags == kModsGmfBorder)
    return launch_policy<PolicyGmfBorder, 256, 2>(kp, st, dc, grid, block, s);
  return launch_variant<PolicyMixedGmf>(kp, st, dc, grid, block, variant, s);
}

cudaError_t occupancy_propagate_mixed_gmf(int dtype, uint32_t flags, int variant, int block,
                                          int* bps) {
  if (variant == 2 && flags == kModsGmfBorder)
    return occupancy_policy<PolicyGmfBorder, 256, 2>(dtype, block, bps);
  return occupancy_variant<PolicyMixedGmf>(dtype, variant, block, bps);
}

cudaError_t sample_field_mixed_gmf(const KParams& kp, const double* xyz, int64_t n, double* B,
                                   cudaStream_t s) {
  return sample_policy<PolicyMixedGmf>(kp, xyz, n, B, s);
}

}  // namespace crp
