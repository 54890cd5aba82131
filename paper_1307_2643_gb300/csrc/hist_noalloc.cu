// hist_noalloc.cu -- the energy histogram of crp_histogram_energy, counted
// into a fixed device array instead of a buffer allocated per call.
//
// For callers that must not allocate device memory during the call: code
// whose device memory is handed out entirely by another allocator, code
// that cannot tolerate an allocation failure part way through a run, or
// code that must not trigger the device-wide synchronisation that freeing
// memory may imply.  The bins live in one file-scope device array of
// CRP_HIST_NOALLOC_MAX_BINS counters, present on every GPU that loads the
// library until the process exits.
#include <math.h>

#include <mutex>

#include "crp_internal.cuh"

namespace crp {
void context_view(const crp_context* c, const int32_t** status, const double** E, uint64_t* n,
                  int* device);
}  // namespace crp

using namespace crp;

namespace {

static __device__ __align__(256) unsigned long long g_noalloc_bins[CRP_HIST_NOALLOC_MAX_BINS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned long long* g_bins_addr[kMaxDevices] = {nullptr};
// One call at a time per device: a call holds its device's lock from the
// clearing of the bins to the end of the copy back, so calls from several
// threads or streams of this process never share the array on the GPU.
std::mutex g_call_mu[kMaxDevices];

__device__ __forceinline__ bool record_selected(int what, int status) {
  switch (what) {
    case CRP_COLLECT_ALL: return true;
    case CRP_COLLECT_FINISHED: return status != CRP_ACTIVE;
    case CRP_COLLECT_DETECTED: return status == CRP_DETECTED;
    case CRP_COLLECT_ACTIVE: return status == CRP_ACTIVE;
    case CRP_COLLECT_AT_BORDER: return status == CRP_AT_BORDER;
  }
  return false;
}

__global__ void k_hist_energy_fixed(const int32_t* status, const double* E, uint64_t n, int what,
                                    double l0, double inv_dl, int nb, unsigned long long* bins) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (!record_selected(what, status[i])) continue;
    const double t = (log(E[i]) - l0) * inv_dl;
    if (!(t >= 0.0) || t >= (double)nb) continue;
    atomicAdd(bins + (int)t, 1ull);
  }
}

// Device address of the fixed bins on `device` (current), looked up once.
crp_status bins_address(int device, unsigned long long** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("crp_histogram_energy_noalloc: device index %d out of range", device);
    return CRP_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_bins_addr[device]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_bins);
    if (e != cudaSuccess) return fail_cuda(e, "crp_histogram_energy_noalloc: cudaGetSymbolAddress");
    g_bins_addr[device] = static_cast<unsigned long long*>(ptr);
  }
  *out = g_bins_addr[device];
  return CRP_OK;
}

}  // namespace

extern "C" crp_status crp_histogram_energy_noalloc(crp_context* ctx, int32_t what, double e_lo,
                                                   double e_hi, int32_t nbins, uint64_t* out,
                                                   void* stream) {
  if (!ctx || !out || !(e_lo > 0.0) || !(e_hi > e_lo) || what < CRP_COLLECT_ALL ||
      what > CRP_COLLECT_AT_BORDER) {
    set_error("crp_histogram_energy_noalloc: bad argument");
    return CRP_E_INVALID;
  }
  if (nbins < 1 || nbins > CRP_HIST_NOALLOC_MAX_BINS) {
    set_error("crp_histogram_energy_noalloc: nbins = %d outside 1..%d (the fixed bin array)",
              nbins, CRP_HIST_NOALLOC_MAX_BINS);
    return CRP_E_INVALID;
  }
  const int32_t* status = nullptr;
  const double* E = nullptr;
  uint64_t n = 0;
  int device = 0;
  context_view(ctx, &status, &E, &n, &device);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) {
    // the symbol address below is per device: resolve it only with the
    // context's device current, never on whatever device a failed switch left
    const cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail_cuda(e, "crp_histogram_energy_noalloc: cudaSetDevice");
  }
  unsigned long long* bins = nullptr;
  crp_status st = bins_address(device, &bins);
  if (st == CRP_OK) {
    std::lock_guard<std::mutex> call_lock(g_call_mu[device]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double l0 = log(e_lo), inv = (double)nbins / (log(e_hi) - l0);
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(unsigned long long) * (size_t)nbins, s);
    if (e == cudaSuccess && n > 0) {
      uint64_t blocks = (n + 255) / 256;
      if (blocks > 65536) blocks = 65536;
      k_hist_energy_fixed<<<(int)blocks, 256, 0, s>>>(status, E, n, what, l0, inv, nbins, bins);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, bins, sizeof(unsigned long long) * (size_t)nbins,
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail_cuda(e, "crp_histogram_energy_noalloc");
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return st;
}
