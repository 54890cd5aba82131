// field.cu -- grid storage and turbulent-field generation.
//
// Storage: one 16-byte float4 (binary32 grids) or 32-byte double (binary64
// grids) per node, components (Bx, By, Bz, 0), x fastest.  A trilinear gather
// then costs one (two) vector loads per corner.
//
// Turbulence (setup, not part of the timed path): Gaussian Fourier modes in
// the band 2pi/lmax <= |k| <= 2pi/lmin, projected perpendicular to k so that
// the field is divergence free, scaled by |k|^(index/2) so that
// |B(k)|^2 ~ |k|^index (Kolmogorov: index = -11/3); the field is the real part
// of the inverse FFT (cuFFT, double complex), with the mean removed and the
// amplitude scaled to the requested B_rms.  The reductions for the mean and
// the rms use fixed-order block partial sums, so the result does not depend
// on scheduling.
#include <cufft.h>
#include <math.h>

#include "crp_internal.cuh"
#include "device_common.cuh"
#include "field_internal.h"

namespace crp {

namespace {

constexpr int kBlock = 256;
constexpr int kRedBlocks = 1024;

__global__ void k_turbulence_modes(int64_t nx, int64_t ny, int64_t nz, double spacing,
                                   double kmin, double kmax, double half_index, uint64_t seed,
                                   double2* out /* 3 component planes of N */) {
  const int64_t N = nx * ny * nz;
  for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < N;
       lin += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = lin % nx, iy = (lin / nx) % ny, iz = lin / (nx * ny);
    out[lin] = make_double2(0.0, 0.0);
    out[N + lin] = make_double2(0.0, 0.0);
    out[2 * N + lin] = make_double2(0.0, 0.0);
    const int64_t mx = ix < (nx + 1) / 2 ? ix : ix - nx;
    const int64_t my = iy < (ny + 1) / 2 ? iy : iy - ny;
    const int64_t mz = iz < (nz + 1) / 2 ? iz : iz - nz;
    const double kx = 2.0 * M_PI * (double)mx / ((double)nx * spacing);
    const double ky = 2.0 * M_PI * (double)my / ((double)ny * spacing);
    const double kz = 2.0 * M_PI * (double)mz / ((double)nz * spacing);
    const double k = sqrt(kx * kx + ky * ky + kz * kz);
    if (!(k >= kmin && k <= kmax)) continue;
    // Nyquist planes stay empty: -k would alias onto a mode whose wavevector
    // is not -k, and the real part would no longer be divergence free.
    if ((nx % 2 == 0 && 2 * ix == nx) || (ny % 2 == 0 && 2 * iy == ny) ||
        (nz % 2 == 0 && 2 * iz == nz))
      continue;
    double re[3], im[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const Philox4 w = draw4(seed, TAG_FIELD, (uint64_t)lin, (uint32_t)c);
      const double u1 = u01_open(w.v0, w.v1);
      const double u2 = u01_open(w.v2, w.v3);
      const double r = sqrt(-2.0 * log(u1));
      double s, co;
      sincospi(2.0 * u2, &s, &co);
      re[c] = r * co;
      im[c] = r * s;
    }
    const double hx = kx / k, hy = ky / k, hz = kz / k;
    const double pr = hx * re[0] + hy * re[1] + hz * re[2];
    const double pi = hx * im[0] + hy * im[1] + hz * im[2];
    re[0] -= pr * hx;
    re[1] -= pr * hy;
    re[2] -= pr * hz;
    im[0] -= pi * hx;
    im[1] -= pi * hy;
    im[2] -= pi * hz;
    const double amp = pow(k, half_index);
    out[lin] = make_double2(re[0] * amp, im[0] * amp);
    out[N + lin] = make_double2(re[1] * amp, im[1] * amp);
    out[2 * N + lin] = make_double2(re[2] * amp, im[2] * amp);
  }
}

// Block partial sums of the real parts (pass 0) or of |B - mean|^2 (pass 1).
__global__ void k_partials(const double2* buf, int64_t N, const double* mean, int pass,
                           double* partial /* [gridDim.x][3] */) {
  __shared__ double sh[3][kBlock];
  double acc[3] = {0.0, 0.0, 0.0};
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = min(N, lo + per);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    if (pass == 0) {
      acc[0] += buf[i].x;
      acc[1] += buf[N + i].x;
      acc[2] += buf[2 * N + i].x;
    } else {
      const double a = buf[i].x - mean[0], b = buf[N + i].x - mean[1], c = buf[2 * N + i].x - mean[2];
      acc[0] += a * a + b * b + c * c;
    }
  }
  for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) partial[blockIdx.x * 3 + c] = sh[c][0];
}

// Fixed-order final sums: out[0..2] = means (pass 0) or out[3] = scale (pass 1).
__global__ void k_finish(const double* partial, int nb, int64_t N, int pass, double brms,
                         double* stats) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nb; ++b)
    for (int c = 0; c < 3; ++c) s[c] += partial[b * 3 + c];
  if (pass == 0) {
    for (int c = 0; c < 3; ++c) stats[c] = s[c] / (double)N;
  } else {
    const double ms = s[0] / (double)N;
    stats[3] = ms > 0.0 ? brms / sqrt(ms) : 0.0;
  }
}

template <class NodeT>
__global__ void k_pack_turbulence(const double2* buf, int64_t N, const double* stats, NodeT* out);

template <>
__global__ void k_pack_turbulence<float4>(const double2* buf, int64_t N, const double* stats,
                                          float4* out) {
  const double m0 = stats[0], m1 = stats[1], m2 = stats[2], sc = stats[3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float4((float)((buf[i].x - m0) * sc), (float)((buf[N + i].x - m1) * sc),
                         (float)((buf[2 * N + i].x - m2) * sc), 0.f);
}

template <>
__global__ void k_pack_turbulence<DNode>(const double2* buf, int64_t N, const double* stats,
                                           DNode* out) {
  const double m0 = stats[0], m1 = stats[1], m2 = stats[2], sc = stats[3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = DNode{(buf[i].x - m0) * sc, (buf[N + i].x - m1) * sc,
                          (buf[2 * N + i].x - m2) * sc, 0.0};
}

template <class SrcT, class NodeT>
__global__ void k_pack_values(const SrcT* src, int64_t N, NodeT* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    NodeT v;
    v.x = src[3 * i];
    v.y = src[3 * i + 1];
    v.z = src[3 * i + 2];
    v.w = 0;
    out[i] = v;
  }
}

template <class NodeT>
__global__ void k_unpack(const NodeT* in, int64_t N, double* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const NodeT v = in[i];
    dst[3 * i] = v.x;
    dst[3 * i + 1] = v.y;
    dst[3 * i + 2] = v.z;
  }
}

int grid_blocks(int64_t N) {
  const int64_t b = (N + kBlock - 1) / kBlock;
  return (int)(b < 65536 ? b : 65536);
}

// Cell (i, j, k) record: the coefficients of the cell's trilinear
// polynomial in the in-cell fractions (tx, ty, tz),
//   B = c0 + c1 tx + c2 ty + c3 tz + c4 tx ty + c5 tx tz + c6 ty tz + c7 tx ty tz,
// from the corner vectors v_(a + 2b + 4c) of nodes (i + a, j + b, k + c)
// (periodic), formed in binary64 and rounded once to binary32; 24 floats
// (coefficient-major, Bx By Bz) in 8 float4, the last two zero.
__global__ void k_grid_cells(const float4* __restrict__ nodes, int64_t nx, int64_t ny, int64_t nz,
                             float4* __restrict__ cells) {
  const int64_t N = nx * ny * nz;
  for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < N;
       lin += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lin % nx, j = (lin / nx) % ny, k = lin / (nx * ny);
    const int64_t i1 = i + 1 == nx ? 0 : i + 1, j1 = j + 1 == ny ? 0 : j + 1,
                  k1 = k + 1 == nz ? 0 : k + 1;
    const int64_t xs[2] = {i, i1}, ys[2] = {j, j1}, zs[2] = {k, k1};
    double v[8][3];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float4 b = nodes[(zs[c >> 2] * ny + ys[(c >> 1) & 1]) * nx + xs[c & 1]];
      v[c][0] = b.x;
      v[c][1] = b.y;
      v[c][2] = b.z;
    }
    float q[32];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double c0 = v[0][d];
      const double c1 = v[1][d] - v[0][d];
      const double c2 = v[2][d] - v[0][d];
      const double c3 = v[4][d] - v[0][d];
      const double c4 = v[3][d] - v[2][d] - v[1][d] + v[0][d];
      const double c5 = v[5][d] - v[4][d] - v[1][d] + v[0][d];
      const double c6 = v[6][d] - v[4][d] - v[2][d] + v[0][d];
      const double c7 = v[7][d] - v[6][d] - v[5][d] - v[3][d] + v[4][d] + v[2][d] + v[1][d] -
                        v[0][d];
      q[d] = (float)c0;
      q[3 + d] = (float)c1;
      q[6 + d] = (float)c2;
      q[9 + d] = (float)c3;
      q[12 + d] = (float)c4;
      q[15 + d] = (float)c5;
      q[18 + d] = (float)c6;
      q[21 + d] = (float)c7;
    }
#pragma unroll
    for (int r = 24; r < 32; ++r) q[r] = 0.f;
    float4* out = cells + 8 * lin;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      out[r] = make_float4(q[4 * r], q[4 * r + 1], q[4 * r + 2], q[4 * r + 3]);
  }
}

}  // namespace

size_t node_bytes(int dtype) { return dtype == CRP_F32 ? sizeof(float4) : sizeof(DNode); }

crp_status grid_cells(const void* nodes, const int64_t n[3], void* cells, cudaStream_t s) {
  const int64_t N = n[0] * n[1] * n[2];
  int64_t g = (N + kBlock - 1) / kBlock;
  if (g > 65535 * 8) g = 65535 * 8;
  k_grid_cells<<<(unsigned)g, kBlock, 0, s>>>(static_cast<const float4*>(nodes), n[0], n[1],
                                               n[2], static_cast<float4*>(cells));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "grid: cell records");
}

crp_status grid_pack(const void* src_dev, int src_dtype, int64_t N, int dtype, void* nodes,
                     cudaStream_t s) {
  const int nb = grid_blocks(N);
  if (src_dtype == CRP_F32 && dtype == CRP_F32)
    k_pack_values<float, float4><<<nb, kBlock, 0, s>>>((const float*)src_dev, N, (float4*)nodes);
  else if (src_dtype == CRP_F32)
    k_pack_values<float, DNode><<<nb, kBlock, 0, s>>>((const float*)src_dev, N, (DNode*)nodes);
  else if (dtype == CRP_F32)
    k_pack_values<double, float4><<<nb, kBlock, 0, s>>>((const double*)src_dev, N, (float4*)nodes);
  else
    k_pack_values<double, DNode><<<nb, kBlock, 0, s>>>((const double*)src_dev, N, (DNode*)nodes);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "grid pack kernel");
}

crp_status grid_unpack(const void* nodes, int dtype, int64_t N, double* dst_dev, cudaStream_t s) {
  const int nb = grid_blocks(N);
  if (dtype == CRP_F32)
    k_unpack<float4><<<nb, kBlock, 0, s>>>((const float4*)nodes, N, dst_dev);
  else
    k_unpack<DNode><<<nb, kBlock, 0, s>>>((const DNode*)nodes, N, dst_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "grid unpack kernel");
}

crp_status grid_turbulence(const crp_grid_desc* d, void* nodes, cudaStream_t s) {
  const int64_t nx = d->n[0], ny = d->n[1], nz = d->n[2];
  const int64_t N = nx * ny * nz;
  const size_t buf_bytes = (size_t)N * 3 * sizeof(double2);
  double2* buf = (double2*)dev_alloc(buf_bytes);
  double* partial = (double*)dev_alloc(kRedBlocks * 3 * sizeof(double) + 4 * sizeof(double));
  if (!buf || !partial) {
    dev_free(buf);
    dev_free(partial);
    set_error("grid_create: out of device memory for the turbulence workspace (%zu bytes)",
              buf_bytes);
    return CRP_E_OOM;
  }
  double* stats = partial + kRedBlocks * 3;
  crp_status st = CRP_OK;
  cufftHandle plan = 0;
  void* work = nullptr;
  do {
    const double kmin = 2.0 * M_PI / d->lmax, kmax = 2.0 * M_PI / d->lmin;
    k_turbulence_modes<<<grid_blocks(N), kBlock, 0, s>>>(nx, ny, nz, d->spacing, kmin, kmax,
                                                         0.5 * d->spectral_index, d->seed, buf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { st = fail_cuda(e, "turbulence modes kernel"); break; }
    // batched 3-D inverse FFT of the three component planes (row-major z, y, x)
    if (cufftCreate(&plan) != CUFFT_SUCCESS) { set_error("cufftCreate failed"); st = CRP_E_CUDA; break; }
    cufftSetAutoAllocation(plan, 0);
    int dims[3] = {(int)nz, (int)ny, (int)nx};
    size_t work_bytes = 0;
    if (cufftMakePlanMany(plan, 3, dims, nullptr, 1, (int)N, nullptr, 1, (int)N, CUFFT_Z2Z, 3,
                          &work_bytes) != CUFFT_SUCCESS) {
      set_error("cufftMakePlanMany failed for %lld x %lld x %lld", (long long)nx, (long long)ny,
                (long long)nz);
      st = CRP_E_CUDA;
      break;
    }
    if (work_bytes) {
      work = dev_alloc(work_bytes);
      if (!work) { set_error("grid_create: out of memory for the FFT work area"); st = CRP_E_OOM; break; }
      cufftSetWorkArea(plan, work);
    }
    cufftSetStream(plan, s);
    if (cufftExecZ2Z(plan, (cufftDoubleComplex*)buf, (cufftDoubleComplex*)buf, CUFFT_INVERSE) !=
        CUFFT_SUCCESS) {
      set_error("cufftExecZ2Z failed");
      st = CRP_E_CUDA;
      break;
    }
    k_partials<<<kRedBlocks, kBlock, 0, s>>>(buf, N, stats, 0, partial);
    k_finish<<<1, 32, 0, s>>>(partial, kRedBlocks, N, 0, d->brms, stats);
    k_partials<<<kRedBlocks, kBlock, 0, s>>>(buf, N, stats, 1, partial);
    k_finish<<<1, 32, 0, s>>>(partial, kRedBlocks, N, 1, d->brms, stats);
    if (d->dtype == CRP_F32)
      k_pack_turbulence<float4><<<grid_blocks(N), kBlock, 0, s>>>(buf, N, stats, (float4*)nodes);
    else
      k_pack_turbulence<DNode><<<grid_blocks(N), kBlock, 0, s>>>(buf, N, stats, (DNode*)nodes);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = fail_cuda(e, "turbulence reduction / pack kernels"); break; }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = fail_cuda(e, "turbulence generation"); break; }
  } while (0);
  if (plan) cufftDestroy(plan);
  dev_free(work);
  dev_free(buf);
  dev_free(partial);
  return st;
}

}  // namespace crp
