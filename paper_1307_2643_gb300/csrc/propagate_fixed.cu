// propagate_fixed.cu -- mixed-precision propagate kernels for the common
// module lists fixed at compile time, in a unit of their own: pair
// production, adiabatic loss, pion production, E_min and observer, with or
// without photodisintegration; and back-tracking through the disk + halo
// field to the galaxy border.  Without the run-time flag tests the unused
// modules' code and registers drop out (no spills at 128 registers); the
// records are byte-identical to the generic kernel's.
#include "propagate_mixed_impl.cuh"

namespace crp {
namespace {

using PolicyEgal = PolicyMixedT<false, false, kModsEgal>;
using PolicyEgalPd = PolicyMixedT<false, false, kModsEgalPd>;
using PolicyGalBorder = PolicyMixedT<true, false, kModsGalBorder>;

}  // namespace

int fixed_modules_index(uint32_t flags) {
  if (flags == kModsEgal) return 0;
  if (flags == kModsEgalPd) return 1;
  if (flags == kModsGalBorder) return 2;
  return -1;
}

cudaError_t launch_propagate_mixed_fixed(int index, const KParams& kp, const DevState& st,
                                         DevCounters* dc, int grid, int block, cudaStream_t s) {
  switch (index) {
    case 0: return launch_policy<PolicyEgal, 256, 2>(kp, st, dc, grid, block, s);
    case 1: return launch_policy<PolicyEgalPd, 256, 2>(kp, st, dc, grid, block, s);
    case 2: return launch_policy<PolicyGalBorder, 256, 2>(kp, st, dc, grid, block, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t occupancy_propagate_mixed_fixed(int index, int dtype, int block, int* bps) {
  switch (index) {
    case 0: return occupancy_policy<PolicyEgal, 256, 2>(dtype, block, bps);
    case 1: return occupancy_policy<PolicyEgalPd, 256, 2>(dtype, block, bps);
    case 2: return occupancy_policy<PolicyGalBorder, 256, 2>(dtype, block, bps);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace crp
