// propagate_gmf.cu -- the mixed-precision propagate kernels with the analytic
// multi-arm galactic field (CRP_GMF), in a unit of their own: the disk + halo
// and plain policies stay free of its code and registers.
#include "propagate_mixed_impl.cuh"

namespace crp {

cudaError_t launch_propagate_mixed_gmf(const KParams& kp, const DevState& st, DevCounters* dc,
                                       int grid, int block, int variant, cudaStream_t s) {
  return launch_variant<PolicyMixedGmf>(kp, st, dc, grid, block, variant, s);
}

cudaError_t occupancy_propagate_mixed_gmf(int dtype, int variant, int block, int* bps) {
  return occupancy_variant<PolicyMixedGmf>(dtype, variant, block, bps);
}

cudaError_t sample_field_mixed_gmf(const KParams& kp, const double* xyz, int64_t n, double* B,
                                   cudaStream_t s) {
  return sample_policy<PolicyMixedGmf>(kp, xyz, n, B, s);
}

}  // namespace crp
