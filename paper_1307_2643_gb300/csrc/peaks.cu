// Measured arithmetic and L2 peaks of the current GPU: the roofline
// denominators the propagation kernels are measured against (binary32 and
// binary64 fused multiply-add issue, and L2-resident read bandwidth).
//
// Each probe is a plain kernel whose work is known exactly:
//   * FMA probes: every thread runs 8 independent multiply-add chains, so
//     the pipe, not the dependency latency, sets the rate (8 chains x 8+
//     warps per scheduler cover the FMA latency many times over);
//   * L2 probe: the grid streams a buffer small enough to stay in L2 (a
//     quarter of the L2 size) several times with 16-byte loads.
// Results feed only a sink word, so nothing is optimised away.
#include <cuda_runtime.h>

#include <cstring>

#include "crp.h"
#include "crp_internal.cuh"

using crp::dev_alloc;
using crp::dev_free;
using crp::fail_cuda;
using crp::set_error;

namespace {

__device__ float g_sink_f;
__device__ double g_sink_d;
__device__ unsigned g_sink_u;

constexpr int kChains = 8;

__global__ void k_fma32(int iters, float seed) {
  float a[kChains];
  const float x = 1.0f - 1e-7f * (float)(threadIdx.x & 7);
  const float y = 1e-8f * (float)(blockIdx.x & 15);
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (float)c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], x, y);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5f) g_sink_f = s;  // practically never; keeps the chains live
}

__global__ void k_fma64(int iters, double seed) {
  double a[kChains];
  const double x = 1.0 - 1e-15 * (double)(threadIdx.x & 7);
  const double y = 1e-17 * (double)(blockIdx.x & 15);
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (double)c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5) g_sink_d = s;
}

__global__ void k_l2_read(const uint4* __restrict__ buf, size_t n16, int passes) {
  unsigned acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);  // L2 only: the probe measures L2, not L1
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  if (acc == 0x9e3779b9u) g_sink_u = acc;
}

}  // namespace

extern "C" crp_status crp_measure_peaks(int32_t device, crp_peaks* out) {
  if (!out) {
    set_error("crp_measure_peaks: out is NULL");
    return CRP_E_INVALID;
  }
  memset(out, 0, sizeof(*out));
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail_cuda(e, "crp_measure_peaks");
  if (device < 0 || device >= ndev) {
    set_error("crp_measure_peaks: device %d not present", device);
    return CRP_E_INVALID;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  int sms = 0, l2 = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  void* buf = nullptr;
  crp_status st = CRP_OK;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const size_t l2_bytes = (size_t)(l2 > 0 ? l2 : (64 << 20)) / 4 / 16 * 16;
  if (e == cudaSuccess) {
    buf = dev_alloc(l2_bytes);
    if (!buf) {
      set_error("crp_measure_peaks: cannot allocate the L2 probe buffer");
      st = CRP_E_OOM;
    }
  }
  if (e == cudaSuccess && st == CRP_OK) e = cudaMemsetAsync(buf, 0x5a, l2_bytes, s);
  // best of three timed launches after one warm-up launch
  auto best_ms = [&](auto launch) -> float {
    float best = 0.f;
    launch();
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
      cudaEventRecord(a, s);
      launch();
      cudaEventRecord(b, s);
      e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    return best;
  };
  if (e == cudaSuccess && st == CRP_OK) {
    const int grid = sms * 8, block = 256;
    const int it32 = 512, it64 = 24;
    const float t32 = best_ms([&] { k_fma32<<<grid, block, 0, s>>>(it32, 0.5f); });
    const float t64 = best_ms([&] { k_fma64<<<grid, block, 0, s>>>(it64, 0.5); });
    const double thr = (double)grid * block * kChains * 16;  // FMAs per iteration
    if (e == cudaSuccess) e = cudaGetLastError();
    if (t32 > 0.f) out->fp32_tflops = 2.0 * thr * it32 / (t32 * 1e-3) / 1e12;
    if (t64 > 0.f) out->fp64_tflops = 2.0 * thr * it64 / (t64 * 1e-3) / 1e12;
    const int passes = 64;
    const size_t n16 = l2_bytes / 16;
    const float tl2 = best_ms([&] {
      k_l2_read<<<sms * 8, 512, 0, s>>>(static_cast<const uint4*>(buf), n16, passes);
    });
    if (e == cudaSuccess) e = cudaGetLastError();
    if (tl2 > 0.f) out->l2_read_gbs = (double)l2_bytes * passes / (tl2 * 1e-3) / 1e9;
    out->sm_count = sms;
    out->l2_bytes = l2;
  }
  if (e != cudaSuccess && st == CRP_OK) st = fail_cuda(e, "crp_measure_peaks");
  if (s) cudaStreamSynchronize(s);
  dev_free(buf);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return st;
}
