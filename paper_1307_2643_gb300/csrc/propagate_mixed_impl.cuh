// propagate_mixed_impl.cuh -- launch, occupancy and field-sampling templates
// of the mixed-precision policies, shared by the units that instantiate them.
#pragma once

#include "propagate.cuh"

namespace crp {

// Register-allocation variants (threads x resident blocks per SM): 2 = 256 x 2
// (128 registers, no spills), 5 = 128 x 5 (96 registers), 3 = 256 x 3 (80).
template <class P>
cudaError_t launch_variant(const KParams& kp, const DevState& st, DevCounters* dc, int grid,
                           int block, int variant, cudaStream_t s) {
  if (variant == 3) return launch_policy<P, 256, 3>(kp, st, dc, grid, block, s);
  if (variant == 5) return launch_policy<P, 128, 5>(kp, st, dc, grid, block, s);
  return launch_policy<P, 256, 2>(kp, st, dc, grid, block, s);
}

template <class P>
cudaError_t occupancy_variant(int dtype, int variant, int block, int* bps) {
  if (variant == 3) return occupancy_policy<P, 256, 3>(dtype, block, bps);
  if (variant == 5) return occupancy_policy<P, 128, 5>(dtype, block, bps);
  return occupancy_policy<P, 256, 2>(dtype, block, bps);
}

template <class Policy, class NodeT>
__global__ void k_sample_mixed(const KParams p, const double* xyz, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    typename Policy::Lane c;
    Policy::init_lane(c);
    c.x[0] = xyz[3 * i];
    c.x[1] = xyz[3 * i + 1];
    c.x[2] = xyz[3 * i + 2];
    Policy::rebase(p, c);
    const float3 B = Policy::template field<NodeT>(p, c, 0.f, 0.f, 0.f);
    out[3 * i] = B.x;
    out[3 * i + 1] = B.y;
    out[3 * i + 2] = B.z;
  }
}

template <class Policy>
cudaError_t sample_policy(const KParams& kp, const double* xyz, int64_t n, double* B,
                          cudaStream_t s) {
  const int64_t g64 = (n + 255) / 256;
  const unsigned g = (unsigned)(g64 < 1 ? 1 : (g64 > 65535 ? 65535 : g64));
  const size_t sm = Policy::kSmemPerThread * 256;
  if (kp.f.dtype == CRP_F32)
    k_sample_mixed<Policy, float4><<<g, 256, sm, s>>>(kp, xyz, n, B);
  else
    k_sample_mixed<Policy, DNode><<<g, 256, sm, s>>>(kp, xyz, n, B);
  return cudaGetLastError();
}

}  // namespace crp
