// propagate_fp64.cu -- binary64 propagate kernels.  Built with -fmad=false:
// every multiply and add is rounded separately, in source order.
#include "propagate.cuh"

namespace crp {

cudaError_t launch_propagate_fp64(const KParams& kp, const DevState& st, DevCounters* dc,
                                  int grid, int block, cudaStream_t s) {
  if (kp.nuc_tab) return launch_propagate_fp64_nuc(kp, st, dc, grid, block, s);
  return launch_policy<PolicyFP64, 128, 2>(kp, st, dc, grid, block, s);
}

cudaError_t occupancy_propagate_fp64(int dtype, int block, int* bps, bool nuc) {
  if (nuc) return occupancy_propagate_fp64_nuc(dtype, block, bps);
  return occupancy_policy<PolicyFP64, 128, 2>(dtype, block, bps);
}

size_t propagate_smem_fp64(int block) { return smem_bytes<PolicyFP64>(block); }

namespace {
template <class NodeT>
__global__ void k_sample_fp64(const KParams p, const double* xyz, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    double B[3];
    field_fp64<NodeT>(p, x, B);
    out[3 * i] = B[0];
    out[3 * i + 1] = B[1];
    out[3 * i + 2] = B[2];
  }
}
}  // namespace

cudaError_t sample_field_fp64(const KParams& kp, const double* xyz, int64_t n, double* B,
                              cudaStream_t s) {
  const int64_t g64 = (n + 255) / 256;
  const unsigned g = (unsigned)(g64 < 1 ? 1 : (g64 > 65535 ? 65535 : g64));
  if (kp.f.dtype == CRP_F32)
    k_sample_fp64<float4><<<g, 256, 0, s>>>(kp, xyz, n, B);
  else
    k_sample_fp64<DNode><<<g, 256, 0, s>>>(kp, xyz, n, B);
  return cudaGetLastError();
}

}  // namespace crp
