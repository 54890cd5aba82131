// mlp.cu -- MLP galactic-lens surrogate: BF16 tensor-core training and
// inference with FP32 accumulation and FP32 master weights.
//
// Network: inputs (n_x, n_y, n_z, log10 R - 19) -> n_hidden ReLU layers of
// width `hidden` -> linear 3-vector, normalised to the predicted direction at
// the galaxy border.  Loss mean(1 - y_hat . t).  Adam (Kingma & Ba 2015) with
// bias correction.  Parameters packed [W1, b1, W2, b2, ...], W_l (n_out, n_in)
// row-major, FP32.
//
// The hidden-to-hidden layers are GEMMs C = A . Bt^T (A: M x K, Bt: N x K,
// both bfloat16 row-major) on the tensor cores (mma.sync m16n8k16, bf16 in,
// f32 accumulate), 128 x 128 x 32 block tiles, double-buffered cp.async
// staging, shared rows padded to 40 elements so fragment loads hit 32
// distinct banks.  Epilogues: bias + ReLU to bf16 (forward), ReLU mask to
// bf16 (backward data), FP32 atomic accumulation (weight gradients, split K
// over the batch).  The thin input (K = 4) and output (N = 3) layers, the
// loss, transposes, bias sums and Adam are plain FP32 kernels.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <utility>
#include <vector>

#include "crp_internal.cuh"
#include "device_common.cuh"
#include "mlp_tc.h"

namespace crp {
void context_pool(const crp_context* c, DevState* st, uint64_t* n, int* device, uint64_t* seed);
}  // namespace crp

using namespace crp;

struct crp_mlp {
  int device;
  int n_in, hidden, n_hidden, n_out;
  int64_t n_params;
  std::vector<int64_t> w_off, b_off;  // offsets of W_l and b_l in the packed vector
  float* params;                      // FP32 master parameters
  float* grad;
  float* m;
  float* v;
  int64_t step;
  std::vector<__nv_bfloat16*> wb, wbt;  // bf16 copies of hidden layers' W and W^T
  std::vector<__nv_bfloat16*> wimg;     // bf16 core-matrix images for the tcgen05 forward
  std::vector<__nv_bfloat16*> wimgT;    // the same images of W^T (one-kernel training step)
  unsigned* tc_err;                     // tcgen05 forward: wait-timeout flag
  int forward_path;                     // CRP_MLP_PATH_*
  int sm_count;
  // batch workspace
  int64_t cap;
  std::vector<__nv_bfloat16*> h;  // activations of each hidden layer [cap][hidden]
  __nv_bfloat16 *dz, *dz2, *dzt, *ht;
  float *y, *dy, *loss;
  // tensor-core training workspace: transposed activations of the layers that
  // feed a hidden GEMM, and transposed backward signals [hidden][tcap] (two,
  // or three for the one-kernel training step)
  int64_t tcap;
  std::vector<__nv_bfloat16*> hT;
  __nv_bfloat16 *dzT, *dzT2, *dzT3;
  // the tensor-core training step as a CUDA graph, replayed with the Adam
  // node's arguments updated.  With the one-kernel step the kernel's node
  // gets each step's x and t as arguments (tg_train); otherwise they are
  // first copied into the fixed staging buffers xs, ts the graph reads
  bool use_graph;
  cudaGraph_t tg_graph;  // the captured graph: its node handles address the exec's nodes
  cudaGraphExec_t tg_exec;
  cudaGraphNode_t tg_adam;
  cudaKernelNodeParams tg_adam_params;
  cudaGraphNode_t tg_train;  // the one-kernel step's node, or null
  cudaKernelNodeParams tg_train_params;
  MlpTrainTcParams tg_train_args;
  TrainStoreMaps tg_train_maps;
  int64_t tg_n;
  cudaStream_t tg_stream;  // private stream the graph is captured on
  float *xs, *ts;
  int64_t scap;
};

namespace {

constexpr int BM = 128, BN = 128, BK = 32, PAD = 40, GEMM_THREADS = 256;

enum Epi { EPI_BIAS_RELU = 0, EPI_MASK = 1, EPI_ATOMIC = 2 };

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (M x N) = A (M x K) . Bt (N x K)^T over k in [k0, k0 + kn).  M, N
// multiples of 128, kn a multiple of 32; blockIdx.z selects the K split.
template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS)
    k_gemm_bf16(const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ Bt,
                int ldb, int K, int splits, const float* __restrict__ bias,
                const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ out_bf,
                float* __restrict__ out_f, int ldc) {
  __shared__ __align__(16) __nv_bfloat16 As[2][BM][PAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][BN][PAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, 64 x 32 each
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kn = K / splits, kbeg = blockIdx.z * kn;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  auto load_tile = [&](int buf, int k) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int chunk = tid + c * GEMM_THREADS;  // 512 chunks of 8 bf16
      const int row = chunk >> 2, col = (chunk & 3) * 8;
      cp_async16(&As[buf][row][col], A + (size_t)(m0 + row) * lda + k + col);
      cp_async16(&Bs[buf][row][col], Bt + (size_t)(n0 + row) * ldb + k + col);
    }
    cp_async_commit();
  };

  const int nk = kn / BK;
  load_tile(0, kbeg);
  for (int it = 0; it < nk; ++it) {
    const int buf = it & 1;
    if (it + 1 < nk) {
      load_tile(buf ^ 1, kbeg + (it + 1) * BK);
      cp_async_wait1();
    } else {
      cp_async_wait0();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int r = wm * 64 + mi * 16 + g;
        af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[buf][r][kk + 2 * t]);
        af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[buf][r + 8][kk + 2 * t]);
        af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[buf][r][kk + 2 * t + 8]);
        af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[buf][r + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn * 32 + ni * 8 + g;
        bf[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[buf][c][kk + 2 * t]);
        bf[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[buf][c][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni]);
    }
    __syncthreads();
  }
  // epilogue: c0,c1 at (row g, cols 2t, 2t+1); c2,c3 at (row g+8, same cols)
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int row = m0 + wm * 64 + mi * 16 + g + half * 8;
        const int col = n0 + wn * 32 + ni * 8 + 2 * t;
        float v0 = acc[mi][ni][2 * half], v1 = acc[mi][ni][2 * half + 1];
        if (EPI == EPI_BIAS_RELU) {
          v0 = fmaxf(v0 + bias[col], 0.f);
          v1 = fmaxf(v1 + bias[col + 1], 0.f);
          *reinterpret_cast<__nv_bfloat162*>(out_bf + (size_t)row * ldc + col) =
              __floats2bfloat162_rn(v0, v1);
        } else if (EPI == EPI_MASK) {
          const __nv_bfloat162 mk =
              *reinterpret_cast<const __nv_bfloat162*>(mask + (size_t)row * ldc + col);
          v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
          v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
          *reinterpret_cast<__nv_bfloat162*>(out_bf + (size_t)row * ldc + col) =
              __floats2bfloat162_rn(v0, v1);
        } else {
          atomicAdd(out_f + (size_t)row * ldc + col, v0);
          atomicAdd(out_f + (size_t)row * ldc + col + 1, v1);
        }
      }
}

// Output layer and loss: y = h W^T + b (one warp per sample); y_hat = y/|y|;
// when t is given, loss += 1 - y_hat.t and dy = -(t - (y_hat.t) y_hat)/|y|/n.
__global__ void k_layer_out(const __nv_bfloat16* __restrict__ h, int64_t n, int hidden,
                            const float* __restrict__ W, const float* __restrict__ b, int n_out,
                            const float* __restrict__ t, float* __restrict__ y_hat,
                            float* __restrict__ dy, float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float lsum = 0.f;  // this warp's loss terms (lane 0)
  for (int64_t r = warp; r < n; r += nw) {
    float y[3] = {0.f, 0.f, 0.f};
    for (int i = lane; i < hidden; i += 32) {
      const float hv = __bfloat162float(h[r * hidden + i]);
      for (int c = 0; c < 3; ++c) y[c] = fmaf(W[c * hidden + i], hv, y[c]);
    }
    for (int c = 0; c < 3; ++c)
      for (int o = 16; o > 0; o >>= 1) y[c] += __shfl_xor_sync(0xffffffffu, y[c], o);
    if (lane == 0) {
      for (int c = 0; c < 3; ++c) y[c] += b[c];
      const float nrm = sqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
      const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
      float yh[3] = {y[0] * inv, y[1] * inv, y[2] * inv};
      if (y_hat)
        for (int c = 0; c < 3; ++c) y_hat[r * 3 + c] = yh[c];
      if (t) {
        const float d = yh[0] * t[r * 3] + yh[1] * t[r * 3 + 1] + yh[2] * t[r * 3 + 2];
        lsum += 1.f - d;
        for (int c = 0; c < 3; ++c)
          dy[r * 3 + c] = -(t[r * 3 + c] - d * yh[c]) * inv / (float)n;
      }
    }
  }
  if (t) {  // one atomic per block
    __shared__ float part[32];
    if (lane == 0) part[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += part[w];
      atomicAdd(loss, b);
    }
  }
}

// ---- generic-shape kernels (any hidden width and input count); the fast
// kernels below cover hidden a multiple of 256 with at most 8 inputs ----
// First layer (K = n_in, small): H1 = bf16(relu(x W1^T + b1)).
__global__ void k_layer_in(const float* __restrict__ x, int n_in, int64_t n,
                           const float* __restrict__ W, const float* __restrict__ b, int hidden,
                           __nv_bfloat16* __restrict__ h) {
  const int64_t total = n * hidden;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / hidden;
    const int o = (int)(e % hidden);
    float acc = b[o];
    for (int i = 0; i < n_in; ++i) acc = fmaf(W[o * n_in + i], x[r * n_in + i], acc);
    h[e] = __float2bfloat16_rn(fmaxf(acc, 0.f));
  }
}

// dH = dy W (per sample, FP32), masked by ReLU of h, to bf16 dz.
__global__ void k_out_backward_data(const float* __restrict__ dy, int64_t n, int hidden,
                                    const float* __restrict__ W, const __nv_bfloat16* __restrict__ h,
                                    __nv_bfloat16* __restrict__ dz) {
  const int64_t total = n * hidden;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / hidden;
    const int i = (int)(e % hidden);
    float v = dy[r * 3] * W[i] + dy[r * 3 + 1] * W[hidden + i] + dy[r * 3 + 2] * W[2 * hidden + i];
    if (!(__bfloat162float(h[e]) > 0.f)) v = 0.f;
    dz[e] = __float2bfloat16_rn(v);
  }
}

// Gradient of a thin layer: dW[o][i] = sum_r dz[r][o] a[r][i], db[o] = sum_r dz[r][o]
// with dz FP32 [n][no] (output layer) or bf16 (input layer), a bf16 [n][ni] or FP32.
template <class DZ, class AT>
__global__ void k_thin_grad(const DZ* __restrict__ dz, int no, const AT* __restrict__ a, int ni,
                            int64_t n, float* __restrict__ dW, float* __restrict__ db) {
  const int o = blockIdx.y, i = blockIdx.z;  // i == ni: bias
  float acc = 0.f;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const float d = (float)dz[r * no + o];
    acc += i < ni ? d * (float)a[r * ni + i] : d;
  }
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if (threadIdx.x == 0) atomicAdd(i < ni ? dW + o * ni + i : db + o, v);
  }
}

// Column sums of a bf16 [n][cols] matrix into FP32 db (atomic).
__global__ void k_colsum(const __nv_bfloat16* __restrict__ z, int64_t n, int cols,
                         float* __restrict__ db) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float acc = 0.f;
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) acc += __bfloat162float(z[r * cols + c]);
  atomicAdd(db + c, acc);
}

// Column moments of a bf16 matrix Z [n][H] (H a multiple of 256) against a
// thin FP32 matrix X [n][NX]: for every column c and i < NX,
//   W[c * wc + i * wi] += sum_r Z[r][c] X[r][i],
// and the bias sums: BX false: b[c] += sum_r Z[r][c]; BX true: b[i] +=
// sum_r X[r][i].  Each warp takes rows r (stride: all warps of the grid) and
// lane l the 8 columns 8 l .. 8 l + 7 of every 256-column group (one 16-byte
// load per row); four rows are loaded before they are used.  The block's
// warps are summed in shared memory and each sum is added once per block.
template <int NX, bool BX>
__global__ void __launch_bounds__(256) k_col_moments(const __nv_bfloat16* __restrict__ Z, int64_t n,
                                                     int H, const float* __restrict__ X,
                                                     float* __restrict__ W, int wc, int wi,
                                                     float* __restrict__ b) {
  constexpr int NQ = NX + 1;  // quantities per column: NX moments and the bias sum
  __shared__ float part[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wstride = (int64_t)gridDim.x * 8;
  for (int cg = 0; cg < H; cg += 256) {
    float acc[8][NQ];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int k = 0; k < NQ; ++k) acc[q][k] = 0.f;
    float xs[NX > 0 ? NX : 1];  // BX: this warp's sums of X (lane 0)
#pragma unroll
    for (int k = 0; k < (NX > 0 ? NX : 1); ++k) xs[k] = 0.f;
    for (int64_t r0 = blockIdx.x * 8 + warp; r0 < n; r0 += 4 * wstride) {
      uint4 zq[4];
      float xv[4][NX > 0 ? NX : 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t r = r0 + u * wstride;
        zq[u] = r < n ? __ldg(reinterpret_cast<const uint4*>(Z + r * H + cg) + lane)
                      : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < NX; ++k) xv[u][k] = r < n ? __ldg(X + r * NX + k) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const __nv_bfloat16* zb = reinterpret_cast<const __nv_bfloat16*>(&zq[u]);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float z = __bfloat162float(zb[q]);
#pragma unroll
          for (int k = 0; k < NX; ++k) acc[q][k] = fmaf(z, xv[u][k], acc[q][k]);
          acc[q][NX] += z;
        }
        if (BX)
#pragma unroll
          for (int k = 0; k < NX; ++k) xs[k] += xv[u][k];
      }
    }
    // block sums, one quantity at a time through shared memory
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      if (BX && k == NX) break;  // the bias comes from X below
#pragma unroll
      for (int q = 0; q < 8; ++q) part[warp][8 * lane + q] = acc[q][k];
      __syncthreads();
      float v = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) v += part[w][threadIdx.x];
      const int c = cg + threadIdx.x;
      if (k < NX)
        atomicAdd(W + (int64_t)c * wc + (int64_t)k * wi, v);
      else
        atomicAdd(b + c, v);
      __syncthreads();
    }
    if (BX && cg == 0) {
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < NX; ++k) part[warp][k] = xs[k];
      __syncthreads();
      if (threadIdx.x < NX) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += part[w][threadIdx.x];
        atomicAdd(b + threadIdx.x, v);
      }
      __syncthreads();
    }
  }
}

// Writes the staged 32-row tile T (32 x 256 bf16 of columns cg ..) into the
// transposed matrix outT [H][n]: thread t writes column cg + t, rows r0 ..
// r0 + 31, as 64 contiguous bytes (rows past n are skipped).
__device__ __forceinline__ void store_tile_transposed(const __nv_bfloat16 (*T)[264], int cg,
                                                      int64_t r0, int64_t n,
                                                      __nv_bfloat16* __restrict__ outT) {
  __nv_bfloat16* dst = outT + (int64_t)(cg + threadIdx.x) * n + r0;
  if (r0 + 32 <= n && n % 8 == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __align__(16) __nv_bfloat16 col[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) col[e] = T[8 * q + e][threadIdx.x];
      reinterpret_cast<uint4*>(dst)[q] = *reinterpret_cast<const uint4*>(col);
    }
  } else {
    for (int rr = 0; rr < 32 && r0 + rr < n; ++rr) dst[rr] = T[rr][threadIdx.x];
  }
}

// First layer, hidden a multiple of 256 and n_in <= 8: h = bf16(relu(W1 x +
// b1)).  A block of 8 warps takes 32 rows, one row per warp at a time; lane l
// computes columns 8 l .. 8 l + 7 of each 256-column group (its weights held
// in registers) and stores them as one 16-byte word.  With hT the tile is
// staged in shared memory and written transposed.
__global__ void __launch_bounds__(256) k_layer_in_tile(const float* __restrict__ x, int n_in,
                                                       int64_t n, const float* __restrict__ W,
                                                       const float* __restrict__ b, int hidden,
                                                       __nv_bfloat16* __restrict__ h,
                                                       __nv_bfloat16* __restrict__ hT) {
  __shared__ __align__(16) __nv_bfloat16 T[32][264];
  __shared__ __align__(16) float sw[9][256];  // this column group's W1 (input-major), then b1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = blockIdx.x * 32ll;
  for (int cg = 0; cg < hidden; cg += 256) {
    // coalesced staging: W1 rows of this group, transposed to input-major
    __syncthreads();
    for (int e = threadIdx.x; e < 256 * n_in; e += 256) {
      const int c = e / n_in, i = e - c * n_in;
      sw[i][c] = W[(int64_t)(cg + c) * n_in + i];
    }
    sw[8][threadIdx.x] = b[cg + threadIdx.x];
    __syncthreads();
    const int c0 = cg + 8 * lane;
    float w[8][8], bb[8];
    {
      const float4 b0 = *reinterpret_cast<const float4*>(&sw[8][8 * lane]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sw[8][8 * lane + 4]);
      bb[0] = b0.x, bb[1] = b0.y, bb[2] = b0.z, bb[3] = b0.w;
      bb[4] = b1.x, bb[5] = b1.y, bb[6] = b1.z, bb[7] = b1.w;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < n_in) {
        const float4 w0 = *reinterpret_cast<const float4*>(&sw[i][8 * lane]);
        const float4 w1 = *reinterpret_cast<const float4*>(&sw[i][8 * lane + 4]);
        w[0][i] = w0.x, w[1][i] = w0.y, w[2][i] = w0.z, w[3][i] = w0.w;
        w[4][i] = w1.x, w[5][i] = w1.y, w[6][i] = w1.z, w[7][i] = w1.w;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q][i] = 0.f;
      }
    }
    for (int rr = warp; rr < 32; rr += 8) {
      const int64_t r = r0 + rr;
      if (r >= n) break;
      float xin[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) xin[i] = i < n_in ? __ldg(x + r * n_in + i) : 0.f;
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float acc = bb[q];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (i < n_in) acc = fmaf(w[q][i], xin[i], acc);
        v[q] = __float2bfloat16_rn(fmaxf(acc, 0.f));
      }
      *reinterpret_cast<uint4*>(h + r * hidden + c0) = *reinterpret_cast<const uint4*>(v);
      if (hT) *reinterpret_cast<uint4*>(&T[rr][8 * lane]) = *reinterpret_cast<const uint4*>(v);
    }
    if (hT) {
      __syncthreads();
      store_tile_transposed(T, cg, r0, n, hT);
      __syncthreads();
    }
  }
}

// Output layer backward, hidden a multiple of 256: dz[r][c] = bf16(dy_r .
// W_out[:, c] where h[r][c] > 0, else 0), tiled as k_layer_in_tile, with dzT
// (when given) written transposed.
__global__ void __launch_bounds__(256) k_out_backward_tile(const float* __restrict__ dy, int64_t n,
                                                           int hidden, const float* __restrict__ W,
                                                           const __nv_bfloat16* __restrict__ h,
                                                           __nv_bfloat16* __restrict__ dz,
                                                           __nv_bfloat16* __restrict__ dzT) {
  __shared__ __align__(16) __nv_bfloat16 T[32][264];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = blockIdx.x * 32ll;
  for (int cg = 0; cg < hidden; cg += 256) {
    const int c0 = cg + 8 * lane;
    float w0[8], w1[8], w2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      w0[q] = __ldg(W + c0 + q);
      w1[q] = __ldg(W + hidden + c0 + q);
      w2[q] = __ldg(W + 2 * hidden + c0 + q);
    }
    for (int rr = warp; rr < 32; rr += 8) {
      const int64_t r = r0 + rr;
      if (r >= n) break;
      const float d0 = __ldg(dy + 3 * r), d1 = __ldg(dy + 3 * r + 1), d2 = __ldg(dy + 3 * r + 2);
      const uint4 hq = __ldg(reinterpret_cast<const uint4*>(h + r * hidden + c0));
      const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&hq);
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float g = d0 * w0[q] + d1 * w1[q] + d2 * w2[q];
        if (!(__bfloat162float(hv[q]) > 0.f)) g = 0.f;
        v[q] = __float2bfloat16_rn(g);
      }
      *reinterpret_cast<uint4*>(dz + r * hidden + c0) = *reinterpret_cast<const uint4*>(v);
      if (dzT) *reinterpret_cast<uint4*>(&T[rr][8 * lane]) = *reinterpret_cast<const uint4*>(v);
    }
    if (dzT) {
      __syncthreads();
      store_tile_transposed(T, cg, r0, n, dzT);
      __syncthreads();
    }
  }
}

// Output layer of a training step in one pass over h = h_{L-1} (hidden 256):
// per row, y = W_out h + b_out (warp sum), y_hat = y / |y|, the loss term
// 1 - y_hat . t and dy = -(t - (y_hat . t) y_hat) / |y| / n; then dz =
// bf16((dy . W_out[:, c]) where h[c] > 0) row-major and transposed, and the
// output layer's gradients dW_out += dy h^T, db_out += dy summed over the
// block's rows.  A block of 8 warps takes 64 rows in tiles of 32, one row per
// warp at a time; lane l owns columns 8 l .. 8 l + 7.
__global__ void __launch_bounds__(256) k_out_layer_train(
    const __nv_bfloat16* __restrict__ h, int64_t n, const float* __restrict__ W,
    const float* __restrict__ bo, const float* __restrict__ t, float* __restrict__ loss,
    __nv_bfloat16* __restrict__ dz, __nv_bfloat16* __restrict__ dzT, float* __restrict__ gW,
    float* __restrict__ gb) {
  constexpr int H = 256;
  __shared__ __align__(16) __nv_bfloat16 T[32][264];
  __shared__ float part[8][H];
  __shared__ float small[8][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = 8 * lane;
  float w0[8], w1[8], w2[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    w0[q] = __ldg(W + c0 + q);
    w1[q] = __ldg(W + H + c0 + q);
    w2[q] = __ldg(W + 2 * H + c0 + q);
  }
  const float b0 = __ldg(bo), b1 = __ldg(bo + 1), b2 = __ldg(bo + 2);
  const float inv_n = 1.f / (float)n;
  float aw0[8], aw1[8], aw2[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) aw0[q] = aw1[q] = aw2[q] = 0.f;
  float ab0 = 0.f, ab1 = 0.f, ab2 = 0.f, lsum = 0.f;
  for (int tile = 0; tile < 2; ++tile) {
    const int64_t r0 = blockIdx.x * 64ll + 32 * tile;
    if (r0 >= n) break;
    for (int rr = warp; rr < 32; rr += 8) {
      const int64_t r = r0 + rr;
      if (r >= n) break;
      const uint4 hq = __ldg(reinterpret_cast<const uint4*>(h + r * H + c0));
      const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&hq);
      float hv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) hv[q] = __bfloat162float(hb[q]);
      float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        y0 = fmaf(w0[q], hv[q], y0);
        y1 = fmaf(w1[q], hv[q], y1);
        y2 = fmaf(w2[q], hv[q], y2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
        y2 += __shfl_xor_sync(0xffffffffu, y2, o);
      }
      y0 += b0;
      y1 += b1;
      y2 += b2;
      const float nrm = sqrtf(y0 * y0 + y1 * y1 + y2 * y2);
      const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
      const float yh0 = y0 * inv, yh1 = y1 * inv, yh2 = y2 * inv;
      const float t0 = __ldg(t + 3 * r), t1 = __ldg(t + 3 * r + 1), t2 = __ldg(t + 3 * r + 2);
      const float d = yh0 * t0 + yh1 * t1 + yh2 * t2;
      const float dy0 = -(t0 - d * yh0) * inv * inv_n;
      const float dy1 = -(t1 - d * yh1) * inv * inv_n;
      const float dy2 = -(t2 - d * yh2) * inv * inv_n;
      if (lane == 0) {
        lsum += 1.f - d;
        ab0 += dy0;
        ab1 += dy1;
        ab2 += dy2;
      }
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float g = dy0 * w0[q] + dy1 * w1[q] + dy2 * w2[q];
        if (!(hv[q] > 0.f)) g = 0.f;
        v[q] = __float2bfloat16_rn(g);
        aw0[q] = fmaf(dy0, hv[q], aw0[q]);
        aw1[q] = fmaf(dy1, hv[q], aw1[q]);
        aw2[q] = fmaf(dy2, hv[q], aw2[q]);
      }
      *reinterpret_cast<uint4*>(dz + r * H + c0) = *reinterpret_cast<const uint4*>(v);
      *reinterpret_cast<uint4*>(&T[rr][c0]) = *reinterpret_cast<const uint4*>(v);
    }
    __syncthreads();
    store_tile_transposed(T, 0, r0, n, dzT);
    __syncthreads();
  }
  // block sums of the gradients, one output at a time through shared memory
  auto block_sum = [&](const float (&a)[8], int o) {
#pragma unroll
    for (int q = 0; q < 8; ++q) part[warp][c0 + q] = a[q];
    __syncthreads();
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += part[w][threadIdx.x];
    atomicAdd(gW + o * H + threadIdx.x, v);
    __syncthreads();
  };
  block_sum(aw0, 0);
  block_sum(aw1, 1);
  block_sum(aw2, 2);
  if (lane == 0) {
    small[warp][0] = ab0;
    small[warp][1] = ab1;
    small[warp][2] = ab2;
    small[warp][3] = lsum;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    float v = 0.f;
    for (int w = 0; w < 8; ++w) v += small[w][threadIdx.x];
    atomicAdd(threadIdx.x < 3 ? gb + threadIdx.x : loss, v);
  }
}

// Transpose a bf16 [rows][cols] matrix into [cols][rows] (32 x 32 tiles).
__global__ void k_transpose(const __nv_bfloat16* __restrict__ in, int64_t rows, int cols,
                            __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int64_t r0 = blockIdx.x * 32ll;
  const int c0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y)
    tile[k][threadIdx.x] = in[(r0 + k) * cols + c0 + threadIdx.x];
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y)
    out[(int64_t)(c0 + k) * rows + r0 + threadIdx.x] = tile[threadIdx.x][k];
}

// bf16 copies W (hidden x hidden) and W^T of a hidden layer, and (when img
// is given) W in the tensor-core operand image of the fused kernels:
// element (o, i) at (o / 8) * (8 n) + (i / 8) * 64 + (o % 8) * 8 + i % 8, and
// W^T in the same image (imgT): element (o, i) of W at
// (i / 8) * (8 n) + (o / 8) * 64 + (i % 8) * 8 + o % 8.
// Index of element (n, k) of an hn x hn bf16 matrix in its tensor-core
// image (the B operand of the tcgen05 kernels): 128-byte-swizzled K-major,
// 64-column blocks of hn rows x 128 bytes, a row's 16-byte chunks XOR-ed with
// the row index mod 8.
__device__ __forceinline__ int64_t img_index(int n, int k, int hn) {
  return (int64_t)(k >> 6) * hn * 64 + n * 64 + ((((k >> 3) & 7) ^ (n & 7)) << 3) + (k & 7);
}

struct Bf16Jobs {
  const float* W[16];
  __nv_bfloat16* wb[16];
  __nv_bfloat16* wbt[16];
  __nv_bfloat16* img[16];
  __nv_bfloat16* imgT[16];
};

// Adam step of one parameter (FP32, bias-corrected moments) from its
// gradient gi and moments mi, vi; returns the new parameter.
__device__ __forceinline__ float adam_one(float pi, float gi, float& mi, float& vi, float lr,
                                          float b1, float b2, float eps, float c1, float c2) {
  mi = b1 * mi + (1.f - b1) * gi;
  vi = b2 * vi + (1.f - b2) * gi * gi;
  return pi - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

constexpr int kAdamTile = 32;  // hidden weights: 32 x 32 tiles, one per block
constexpr int kAdamRest = 64;  // blocks for the other parameters
int adam_blocks(int nj, int hn) { return nj * (hn / kAdamTile) * (hn / kAdamTile) + kAdamRest; }

// Adam step of every parameter; a parameter of a hidden weight matrix
// (nj jobs, hn x hn each, hn a multiple of 32, in ascending address order)
// also goes to that layer's bf16 copies and images, so no separate
// conversion pass follows the step.  The first nj (hn / 32)^2 blocks (256
// threads) each take a 32 x 32 tile of one matrix: all loads first, then
// coalesced updates and row-major copies, then the transposed copies from
// the tile staged in shared memory; the last kAdamRest blocks take the other
// parameters (the ranges between the matrices).
__global__ void __launch_bounds__(256)
    k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
           float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
           float c2, const Bf16Jobs jobs, int nj, int hn) {
  const int tpr = hn / kAdamTile;  // tiles per row of a matrix
  const int tiles = nj * tpr * tpr;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t nn = (int64_t)hn * hn;
  if ((int)blockIdx.x < tiles) {
    constexpr int R = kAdamTile / 8;  // rows of the tile per thread
    __shared__ __nv_bfloat16 tile[kAdamTile][kAdamTile + 2];
    const int j = blockIdx.x / (tpr * tpr), tb = blockIdx.x % (tpr * tpr);
    const int o0 = (tb / tpr) * kAdamTile, i0 = (tb % tpr) * kAdamTile;
    const int64_t base = jobs.W[j] - p;
    __nv_bfloat16 *wb = jobs.wb[j], *wbt = jobs.wbt[j], *img = jobs.img[j], *imgT = jobs.imgT[j];
    float pv[R], gv[R], mv[R], vv[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int64_t i = base + (int64_t)(o0 + ty + 8 * k) * hn + i0 + tx;
      pv[k] = p[i];
      gv[k] = g[i];
      mv[k] = m[i];
      vv[k] = v[i];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int o = o0 + ty + 8 * k, ii = i0 + tx;
      const int64_t e = (int64_t)o * hn + ii;
      const float pi = adam_one(pv[k], gv[k], mv[k], vv[k], lr, b1, b2, eps, c1, c2);
      p[base + e] = pi;
      m[base + e] = mv[k];
      v[base + e] = vv[k];
      const __nv_bfloat16 bv = __float2bfloat16_rn(pi);
      wb[e] = bv;
      if (img) img[img_index(o, ii, hn)] = bv;
      tile[ty + 8 * k][tx] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R; ++k) {
      // element (o, ii) = (o0 + tx, i0 + ty + 8 k): consecutive lanes, consecutive o
      const int o = o0 + tx, ii = i0 + ty + 8 * k;
      const __nv_bfloat16 bv = tile[tx][ty + 8 * k];
      wbt[(int64_t)ii * hn + o] = bv;
      if (imgT) imgT[img_index(ii, o, hn)] = bv;
    }
    return;
  }
  // parameter c of the ones outside the matrices -> its index (the matrices
  // are skipped in ascending order)
  const int64_t nrest = n - (int64_t)nj * nn;
  const int64_t stride = (int64_t)(gridDim.x - tiles) * blockDim.x;
  for (int64_t c = (int64_t)(blockIdx.x - tiles) * blockDim.x + threadIdx.x; c < nrest;
       c += stride) {
    int64_t i = c;
    for (int jj = 0; jj < nj; ++jj)
      if (i >= jobs.W[jj] - p) i += nn;
    float mi = m[i], vi = v[i];
    p[i] = adam_one(p[i], g[i], mi, vi, lr, b1, b2, eps, c1, c2);
    m[i] = mi;
    v[i] = vi;
  }
}

__global__ void k_to_bf16_pair(const Bf16Jobs jobs, int n) {
  const float* __restrict__ W = jobs.W[blockIdx.y];
  __nv_bfloat16* __restrict__ wb = jobs.wb[blockIdx.y];
  __nv_bfloat16* __restrict__ wbt = jobs.wbt[blockIdx.y];
  __nv_bfloat16* __restrict__ img = jobs.img[blockIdx.y];
  __nv_bfloat16* __restrict__ imgT = jobs.imgT[blockIdx.y];
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(e / n), i = (int)(e % n);
    const __nv_bfloat16 v = __float2bfloat16_rn(W[e]);
    wb[e] = v;
    wbt[(int64_t)i * n + o] = v;
    if (img) img[img_index(o, i, n)] = v;
    if (imgT) imgT[img_index(i, o, n)] = v;
  }
}

// He-normal initialisation from Philox (tag 4, id = parameter index):
// W ~ N(0, 2 / fan_in) for ReLU layers, N(0, 1 / fan_in) for the output.
__global__ void k_init(float* p, int64_t n, const int64_t* off, const int* fan_in, const int* kind,
                       int n_layers, uint64_t seed) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < n_layers * 2 && off[l + 1] <= k) ++l;
    if (kind[l] == 1) {  // bias
      p[k] = 0.f;
      continue;
    }
    const Philox4 w = draw4(seed, 4u, (uint64_t)k, 0u);
    const double u1 = u01_open(w.v0, w.v1), u2 = u01_open(w.v2, w.v3);
    const double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    const double var = (l / 2 == n_layers - 1 ? 1.0 : 2.0) / (double)fan_in[l];
    p[k] = (float)(z * sqrt(var));
  }
}

int nblk(int64_t n, int b) {
  const int64_t g = (n + b - 1) / b;
  return (int)(g < 1 ? 1 : (g > 65536 ? 65536 : g));
}

void free_ws(crp_mlp* M) {
  for (auto* p : M->h) dev_free(p);
  M->h.clear();
  dev_free(M->dz);
  dev_free(M->dz2);
  dev_free(M->dzt);
  dev_free(M->ht);
  dev_free(M->y);
  dev_free(M->dy);
  dev_free(M->loss);
  M->dz = M->dz2 = M->dzt = M->ht = nullptr;
  M->y = M->dy = M->loss = nullptr;
  M->cap = 0;
}

void free_tws(crp_mlp* M) {
  for (auto* p : M->hT) dev_free(p);
  M->hT.clear();
  dev_free(M->dzT);
  dev_free(M->dzT2);
  dev_free(M->dzT3);
  M->dzT = M->dzT2 = M->dzT3 = nullptr;
  M->tcap = 0;
}

void drop_graph(crp_mlp* M) {
  if (M->tg_exec) cudaGraphExecDestroy(M->tg_exec);
  if (M->tg_graph) cudaGraphDestroy(M->tg_graph);
  M->tg_exec = nullptr;
  M->tg_graph = nullptr;
  M->tg_adam = nullptr;
  M->tg_train = nullptr;
  M->tg_n = 0;
}

// Staging buffers of the graph-replayed training step.
crp_status ensure_stage(crp_mlp* M, int64_t n) {
  if (M->scap >= n) return CRP_OK;
  drop_graph(M);
  dev_free(M->xs);
  dev_free(M->ts);
  M->xs = static_cast<float*>(dev_alloc(sizeof(float) * (size_t)n * M->n_in));
  M->ts = static_cast<float*>(dev_alloc(sizeof(float) * (size_t)n * 3));
  if (!M->xs || !M->ts) {
    dev_free(M->xs);
    dev_free(M->ts);
    M->xs = M->ts = nullptr;
    M->scap = 0;
    set_error("mlp: cannot allocate the training staging buffers");
    return CRP_E_OOM;
  }
  M->scap = n;
  return CRP_OK;
}

// The one-kernel training step applies: the tensor-core shapes with three
// hidden-to-hidden layers (the surrogate's 4 x 256).
bool train_fused_ok(const crp_mlp* M) {
  return !M->wimg.empty() && M->hidden == 256 && M->n_hidden - 1 == kMlpTrainGemm;
}

// Transposed activations for the tensor-core training step (allocated only
// when training on that path).
crp_status ensure_tws(crp_mlp* M, int64_t n) {
  if (M->tcap >= n) return CRP_OK;
  drop_graph(M);
  free_tws(M);
  const size_t hb = sizeof(__nv_bfloat16) * (size_t)n * M->hidden;
  for (int l = 0; l + 1 < M->n_hidden; ++l)
    M->hT.push_back(static_cast<__nv_bfloat16*>(dev_alloc(hb)));
  M->dzT = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  M->dzT2 = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  if (train_fused_ok(M)) M->dzT3 = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  bool ok = M->dzT && M->dzT2 && (M->dzT3 || !train_fused_ok(M));
  for (auto* p : M->hT) ok = ok && p;
  if (!ok) {
    free_tws(M);
    set_error("mlp: cannot allocate the training workspace for %lld samples", (long long)n);
    return CRP_E_OOM;
  }
  M->tcap = n;
  return CRP_OK;
}

crp_status ensure_ws(crp_mlp* M, int64_t n) {
  if (M->cap >= n) return CRP_OK;
  drop_graph(M);
  free_ws(M);
  const size_t hb = sizeof(__nv_bfloat16) * (size_t)n * M->hidden;
  for (int l = 0; l < M->n_hidden; ++l) M->h.push_back(static_cast<__nv_bfloat16*>(dev_alloc(hb)));
  M->dz = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  M->dz2 = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  M->dzt = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  M->ht = static_cast<__nv_bfloat16*>(dev_alloc(hb));
  M->y = static_cast<float*>(dev_alloc(sizeof(float) * 3 * n));
  M->dy = static_cast<float*>(dev_alloc(sizeof(float) * 3 * n));
  M->loss = static_cast<float*>(dev_alloc(sizeof(float)));
  bool ok = M->dz && M->dz2 && M->dzt && M->ht && M->y && M->dy && M->loss;
  for (auto* p : M->h) ok = ok && p;
  if (!ok) {
    free_ws(M);
    set_error("mlp: cannot allocate the workspace for %lld samples", (long long)n);
    return CRP_E_OOM;
  }
  M->cap = n;
  return CRP_OK;
}

// The bf16 conversion jobs of the hidden layers (at most 16); returns their count.
int bf16_jobs(const crp_mlp* M, Bf16Jobs* jobs) {
  memset(jobs, 0, sizeof(*jobs));
  int nj = 0;
  for (int l = 1; l < M->n_hidden && nj < 16; ++l, ++nj) {
    jobs->W[nj] = M->params + M->w_off[l];
    jobs->wb[nj] = M->wb[l];
    jobs->wbt[nj] = M->wbt[l];
    jobs->img[nj] = M->wimg.empty() ? nullptr : M->wimg[l];
    jobs->imgT[nj] = M->wimgT.empty() ? nullptr : M->wimgT[l];
  }
  return nj;
}

crp_status refresh_bf16(crp_mlp* M, cudaStream_t s) {
  // every hidden layer in one launch (grid.y = layer), up to 16 layers
  Bf16Jobs jobs;
  const int nj = bf16_jobs(M, &jobs);
  if (nj > 0) {
    const int64_t total = (int64_t)M->hidden * M->hidden;
    const unsigned gx = (unsigned)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    k_to_bf16_pair<<<dim3(gx, nj), 256, 0, s>>>(jobs, M->hidden);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "mlp: bf16 weights");
}

// Launchers of the thin layers: the tiled / column-moment kernels when the
// hidden width is a multiple of 256 and there are at most 8 inputs (the
// surrogate's shape, and every shape the tensor-core path takes), the
// generic kernels otherwise.
bool fast_shape(const crp_mlp* M) { return M->hidden % 256 == 0 && M->n_in <= 8; }

unsigned red_blocks(const crp_mlp* M) {
  return (unsigned)(2 * (M->sm_count > 0 ? M->sm_count : 152));
}

void launch_layer_in(crp_mlp* M, const float* x, int64_t n, __nv_bfloat16* hT, cudaStream_t s) {
  const float* W = M->params + M->w_off[0];
  const float* b = M->params + M->b_off[0];
  if (fast_shape(M))
    k_layer_in_tile<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(x, M->n_in, n, W, b, M->hidden,
                                                               M->h[0], hT);
  else
    k_layer_in<<<nblk(n * M->hidden, 256), 256, 0, s>>>(x, M->n_in, n, W, b, M->hidden, M->h[0]);
}

void launch_out_backward(crp_mlp* M, int64_t n, __nv_bfloat16* dzT, cudaStream_t s) {
  const int L = M->n_hidden, H = M->hidden;
  const float* W = M->params + M->w_off[L];
  if (fast_shape(M))
    k_out_backward_tile<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(M->dy, n, H, W, M->h[L - 1],
                                                                   M->dz, dzT);
  else
    k_out_backward_data<<<nblk(n * H, 256), 256, 0, s>>>(M->dy, n, H, W, M->h[L - 1], M->dz);
}

// db += column sums of dz (a hidden layer's bias gradient)
void launch_colsum(crp_mlp* M, const __nv_bfloat16* dz, int64_t n, float* db, cudaStream_t s) {
  const int H = M->hidden;
  if (fast_shape(M))
    k_col_moments<0, false><<<red_blocks(M), 256, 0, s>>>(dz, n, H, nullptr, nullptr, 0, 0, db);
  else
    k_colsum<<<dim3(256, (H + 255) / 256), 256, 0, s>>>(dz, n, H, db);
}

// output layer: dW_out[o][c] = sum_r dy[r][o] h[r][c], db_out[o] = sum_r dy[r][o]
void launch_grad_out(crp_mlp* M, int64_t n, cudaStream_t s) {
  const int L = M->n_hidden, H = M->hidden;
  float* gW = M->grad + M->w_off[L];
  float* gb = M->grad + M->b_off[L];
  if (fast_shape(M))
    k_col_moments<3, true><<<red_blocks(M), 256, 0, s>>>(M->h[L - 1], n, H, M->dy, gW, 1, H, gb);
  else
    k_thin_grad<float, __nv_bfloat16><<<dim3(64, 3, H + 1), 256, 0, s>>>(M->dy, 3, M->h[L - 1], H,
                                                                        n, gW, gb);
}

// input layer: dW1[c][i] = sum_r dz[r][c] x[r][i], db1[c] = sum_r dz[r][c]
void launch_grad_in(crp_mlp* M, const __nv_bfloat16* dz, const float* x, int64_t n,
                    cudaStream_t s) {
  const int H = M->hidden, ni = M->n_in;
  float* gW = M->grad + M->w_off[0];
  float* gb = M->grad + M->b_off[0];
  if (!fast_shape(M)) {
    k_thin_grad<__nv_bfloat16, float><<<dim3(64, H, ni + 1), 256, 0, s>>>(dz, H, x, ni, n, gW, gb);
    return;
  }
  const unsigned g = red_blocks(M);
  switch (ni) {
#define CRP_GRAD_IN(NI)                                                                  \
  case NI:                                                                               \
    k_col_moments<NI, false><<<g, 256, 0, s>>>(dz, n, H, x, gW, ni, 1, gb);              \
    break;
    CRP_GRAD_IN(1)
    CRP_GRAD_IN(2)
    CRP_GRAD_IN(3)
    CRP_GRAD_IN(4)
    CRP_GRAD_IN(5)
    CRP_GRAD_IN(6)
    CRP_GRAD_IN(7)
    CRP_GRAD_IN(8)
#undef CRP_GRAD_IN
    default:
      break;
  }
}

template <int EPI>
void gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bt, int ldb, int64_t M, int N, int K,
          int splits, const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out_bf,
          float* out_f, int ldc, cudaStream_t s) {
  dim3 grid((unsigned)(M / BM), (unsigned)(N / BN), (unsigned)splits);
  k_gemm_bf16<EPI><<<grid, GEMM_THREADS, 0, s>>>(A, lda, Bt, ldb, K, splits, bias, mask, out_bf,
                                                 out_f, ldc);
}

// Forward over n samples (n a multiple of 128): activations in M->h, the
// normalised output in y_hat; with targets, the loss and dy as well.  tc: the
// hidden GEMMs on the tensor cores (tcgen05), also writing the transposed
// activations the weight gradients need; else the layered mma.sync GEMMs.
crp_status forward(crp_mlp* M, const float* x, int64_t n, const float* t, float* y_hat,
                   cudaStream_t s, bool tc = false) {
  // training on the tensor-core path: the output layer (loss, dy and its
  // backward) runs fused at the start of backward()
  const bool fused_out = tc && t && !y_hat && M->hidden == 256;
  const int H = M->hidden;
  if (fused_out) {
    // every hidden layer in one persistent tcgen05 kernel, storing each
    // activation and the transposes the weight gradients read
    MlpTcParams P;
    memset(&P, 0, sizeof(P));
    P.x = x;
    P.n_in = M->n_in;
    P.n_gemm = M->n_hidden - 1;
    P.n_tiles = n / 128;
    P.W1 = M->params + M->w_off[0];
    P.b1 = M->params + M->b_off[0];
    for (int l = 1; l < M->n_hidden; ++l) {
      P.Wimg[l - 1] = M->wimg[l];
      P.bh[l - 1] = M->params + M->b_off[l];
    }
    P.Wout = M->params + M->w_off[M->n_hidden];  // staged by the kernel, unused here
    P.bout = M->params + M->b_off[M->n_hidden];
    for (int l = 0; l < M->n_hidden; ++l) {
      P.h[l] = M->h[l];
      P.hT[l] = l + 1 < M->n_hidden ? M->hT[l] : nullptr;
    }
    P.ldt = n;
    P.err = M->tc_err;
    cudaError_t e = cudaMemsetAsync(M->loss, 0, sizeof(float), s);
    if (e == cudaSuccess) e = mlp_forward_tc_train(P, M->sm_count, s);
    return e == cudaSuccess ? CRP_OK : fail_cuda(e, "mlp: tensor-core training forward");
  }
  launch_layer_in(M, x, n, tc ? M->hT[0] : nullptr, s);
  for (int l = 1; l < M->n_hidden; ++l) {
    if (tc) {
      GemmTcParams g;
      memset(&g, 0, sizeof(g));
      g.A = M->h[l - 1];
      g.lda = H;
      g.B = M->wb[l];
      g.ldb = H;
      g.M = n;
      g.K = H;
      g.splits = 1;
      g.bias = M->params + M->b_off[l];
      g.out = M->h[l];
      g.ldo = H;
      g.out_t = l + 1 < M->n_hidden ? M->hT[l] : nullptr;  // feeds the next layer's dW
      g.ldot = n;
      g.err = M->tc_err;
      const cudaError_t e = gemm_tc(GEMM_TC_BIAS_RELU, g, M->device, M->sm_count, s);
      if (e != cudaSuccess) return fail_cuda(e, "mlp: tensor-core forward GEMM");
    } else {
      gemm<EPI_BIAS_RELU>(M->h[l - 1], H, M->wb[l], H, n, H, H, 1, M->params + M->b_off[l],
                          nullptr, M->h[l], nullptr, H, s);
    }
  }
  const int lo = M->n_hidden;
  if (t) cudaMemsetAsync(M->loss, 0, sizeof(float), s);
  if (!fused_out)
    k_layer_out<<<nblk(n * 32, 256), 256, 0, s>>>(M->h[lo - 1], n, H, M->params + M->w_off[lo],
                                                  M->params + M->b_off[lo], 3, t, y_hat, M->dy,
                                                  M->loss);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "mlp: forward");
}

// Backward over the batch of the last forward: gradients (FP32, summed over
// the batch) of every parameter into M->grad.  tc: weight gradients and
// backward-data products on the tensor cores, reading the transposed signals
// the epilogues wrote; else transposes plus the layered mma.sync GEMMs.
crp_status backward(crp_mlp* M, const float* x, const float* t, int64_t n, cudaStream_t s,
                    bool tc = false) {
  const int H = M->hidden, L = M->n_hidden;
  cudaMemsetAsync(M->grad, 0, sizeof(float) * M->n_params, s);
  // output layer
  if (tc && H == 256) {  // forward() left the output layer to this fused pass
    k_out_layer_train<<<(unsigned)((n + 63) / 64), 256, 0, s>>>(
        M->h[L - 1], n, M->params + M->w_off[L], M->params + M->b_off[L], t, M->loss, M->dz,
        M->dzT, M->grad + M->w_off[L], M->grad + M->b_off[L]);
  } else {
    launch_grad_out(M, n, s);
    launch_out_backward(M, n, tc ? M->dzT : nullptr, s);
  }
  __nv_bfloat16* dz = M->dz;
  __nv_bfloat16* dz_next = M->dz2;
  __nv_bfloat16* dzT = M->dzT;
  __nv_bfloat16* dzT_next = M->dzT2;
  const int splits = n >= 128 * 64 ? 32 : (int)(n / 128 < 1 ? 1 : n / 128);
  for (int l = L - 1; l >= 1; --l) {
    // W_l maps h[l-1] -> h[l]; dz holds dL/dz_l (bf16, [n][H])
    if (tc) {
      GemmTcParams g;
      memset(&g, 0, sizeof(g));
      g.err = M->tc_err;
      // dW_l += dz_l^T h_{l-1}: A = dz_l^T [H][n], B = h_{l-1}^T [H][n], K = n split
      g.A = dzT;
      g.lda = n;
      g.B = M->hT[l - 1];
      g.ldb = n;
      g.M = H;
      g.K = n;
      const int64_t sp = n / 256 < 1 ? 1 : n / 256;
      const int64_t sp_max = M->sm_count / 2 > 1 ? M->sm_count / 2 : 1;
      g.splits = (int)(sp < sp_max ? sp : sp_max);
      g.out_f = M->grad + M->w_off[l];
      g.ldf = H;
      g.rowsum = M->grad + M->b_off[l];  // db_l: the rows of dz_l^T summed over the batch
      cudaError_t e = gemm_tc(GEMM_TC_ATOMIC, g, M->device, M->sm_count, s);
      if (e != cudaSuccess) return fail_cuda(e, "mlp: tensor-core weight-gradient GEMM");
      // dz_{l-1} = (dz_l W_l) masked by ReLU'(h_{l-1}): B = W_l^T [H][H]
      memset(&g, 0, sizeof(g));
      g.err = M->tc_err;
      g.A = dz;
      g.lda = H;
      g.B = M->wbt[l];
      g.ldb = H;
      g.M = n;
      g.K = H;
      g.splits = 1;
      g.mask = M->h[l - 1];
      g.ldm = H;
      g.out = dz_next;
      g.ldo = H;
      g.out_t = l > 1 ? dzT_next : nullptr;
      g.ldot = n;
      if (l == 1) {  // dz_0 feeds only the input layer's gradients: taken in this epilogue
        g.xin = x;
        g.n_in = M->n_in;
        g.gw_in = M->grad + M->w_off[0];
        g.gb_in = M->grad + M->b_off[0];
      }
      e = gemm_tc(GEMM_TC_MASK, g, M->device, M->sm_count, s);
      if (e != cudaSuccess) return fail_cuda(e, "mlp: tensor-core backward-data GEMM");
    } else {
      const dim3 tb(32, 8);
      k_transpose<<<dim3((unsigned)(n / 32), H / 32), tb, 0, s>>>(dz, n, H, M->dzt);
      k_transpose<<<dim3((unsigned)(n / 32), H / 32), tb, 0, s>>>(M->h[l - 1], n, H, M->ht);
      int sp = splits;
      while (sp > 1 && (n / sp) % BK != 0) --sp;
      gemm<EPI_ATOMIC>(M->dzt, (int)n, M->ht, (int)n, H, H, (int)n, sp, nullptr, nullptr, nullptr,
                       M->grad + M->w_off[l], H, s);
      launch_colsum(M, dz, n, M->grad + M->b_off[l], s);
      gemm<EPI_MASK>(dz, H, M->wbt[l], H, n, H, H, 1, nullptr, M->h[l - 1], dz_next, nullptr, H, s);
    }
    std::swap(dz, dz_next);
    std::swap(dzT, dzT_next);
  }
  // input layer: dz holds dL/dz_1 (on the tensor-core path the last
  // backward-data GEMM has already added its gradients)
  if (!tc) launch_grad_in(M, dz, x, n, s);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "mlp: backward");
}

// Gradients of one training step on the tensor cores with the per-sample work
// in one kernel (forward, output layer and loss, backward signals, the input
// and output layers' gradients), then the hidden layers' weight gradients
// dW_l = dz_l^T h_{l-1} and bias sums as split-K GEMMs over the activations
// and signals that kernel wrote (row-major, in the transposed-activation
// workspace of the layered path, which has the same size).
crp_status train_fused(crp_mlp* M, const float* x, const float* t, int64_t n, cudaStream_t s) {
  const int H = M->hidden, L = M->n_hidden;
  cudaError_t e = cudaMemsetAsync(M->grad, 0, sizeof(float) * M->n_params, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->loss, 0, sizeof(float), s);
  MlpTrainTcParams P;
  memset(&P, 0, sizeof(P));
  P.x = x;
  P.t = t;
  P.n_in = M->n_in;
  P.n = n;
  P.n_tiles = n / 128;
  P.W1 = M->params + M->w_off[0];
  P.b1 = M->params + M->b_off[0];
  for (int l = 1; l < L; ++l) {
    P.Wimg[l - 1] = M->wimg[l];
    P.WimgT[l - 1] = M->wimgT[l];
    P.bh[l - 1] = M->params + M->b_off[l];
  }
  P.Wout = M->params + M->w_off[L];
  P.bout = M->params + M->b_off[L];
  for (int l = 0; l + 1 < L; ++l) P.h[l] = M->hT[l];
  __nv_bfloat16* sig[kMlpTrainGemm] = {M->dzT, M->dzT2, M->dzT3};
  for (int l = L - 1, k = 0; l >= 1; --l, ++k) P.dz[l] = sig[k];
  P.loss = M->loss;
  P.gW1 = M->grad + M->w_off[0];
  P.gb1 = M->grad + M->b_off[0];
  P.gWout = M->grad + M->w_off[L];
  P.gbout = M->grad + M->b_off[L];
  P.err = M->tc_err;
  if (e == cudaSuccess) e = mlp_train_tc(P, M->sm_count, s);
  if (e != cudaSuccess) return fail_cuda(e, "mlp: tensor-core training kernel");
  // the layers' weight gradients are independent: one launch for all three
  GemmTcParams gs[kMlpTrainGemm];
  int ng = 0;
  for (int l = L - 1; l >= 1; --l) {
    // dW_l += dz_l^T h_{l-1}: A = dz_l [n][H], B = h_{l-1} [n][H], K = n split
    GemmTcParams& g = gs[ng++];
    memset(&g, 0, sizeof(g));
    g.err = M->tc_err;
    g.A = P.dz[l];
    g.lda = H;
    g.B = P.h[l - 1];
    g.ldb = H;
    g.M = H;
    g.K = n;
    const int64_t sp = n / 256 < 1 ? 1 : n / 256;
    const int64_t sp_max = M->sm_count / 2 > 1 ? M->sm_count / 2 : 1;
    g.splits = (int)(sp < sp_max ? sp : sp_max);
    g.out_f = M->grad + M->w_off[l];
    g.ldf = H;
    g.rowsum = M->grad + M->b_off[l];  // db_l: the columns of dz_l summed over the batch
  }
  e = wgrad_tc(gs, ng, M->sm_count, s);
  if (e != cudaSuccess) return fail_cuda(e, "mlp: tensor-core weight-gradient GEMMs");
  return CRP_OK;
}

// Gradients of one training step: the one-kernel form where it applies, else
// the forward and backward passes.
crp_status step_gradients(crp_mlp* M, const float* x, const float* t, int64_t n, cudaStream_t s,
                          bool tc) {
  if (tc && train_fused_ok(M)) return train_fused(M, x, t, n, s);
  crp_status st = forward(M, x, n, t, nullptr, s, tc);
  if (st == CRP_OK) st = backward(M, x, t, n, s, tc);
  return st;
}

// Record the tensor-core training step of n samples (reading the staging
// buffers) as a graph on the private stream; nothing runs.  Any failure
// leaves the step eager (and clears the error state it raised).
void capture_train_graph(crp_mlp* M, int64_t n) {
  drop_graph(M);
  if (!M->tg_stream && cudaStreamCreateWithFlags(&M->tg_stream, cudaStreamNonBlocking) != cudaSuccess) {
    M->tg_stream = nullptr;
    cudaGetLastError();
    return;
  }
  cudaStream_t cs = M->tg_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  crp_status st = step_gradients(M, M->xs, M->ts, n, cs, true);
  if (st == CRP_OK) {
    Bf16Jobs jobs;
    const int nj = bf16_jobs(M, &jobs);
    k_adam<<<adam_blocks(nj, M->hidden), 256, 0, cs>>>(M->params, M->grad, M->m, M->v,
                                                       M->n_params, 0.f, 0.9f, 0.999f, 1e-8f, 1.f,
                                                       1.f, jobs, nj, M->hidden);
    if (cudaGetLastError() != cudaSuccess) st = CRP_E_CUDA;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &g);
  cudaGraphNode_t adam = nullptr, train = nullptr;
  cudaKernelNodeParams ap, tp;
  memset(&ap, 0, sizeof(ap));
  memset(&tp, 0, sizeof(tp));
  const void* train_fn = train_fused_ok(M) ? mlp_train_tc_kernel(M->n_in) : nullptr;
  if (st == CRP_OK && ec == cudaSuccess && g) {
    size_t count = 0;
    cudaGraphGetNodes(g, nullptr, &count);
    std::vector<cudaGraphNode_t> nodes(count);
    if (count && cudaGraphGetNodes(g, nodes.data(), &count) == cudaSuccess) {
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p;
        if (cudaGraphKernelNodeGetParams(nd, &p) != cudaSuccess) continue;
        if (p.func == reinterpret_cast<void*>(k_adam)) {
          adam = nd;
          ap = p;
        } else if (train_fn && p.func == train_fn && p.kernelParams) {
          // the launch's arguments, kept to be re-sent with each step's x, t
          train = nd;
          tp = p;
          memcpy(&M->tg_train_args, p.kernelParams[0], sizeof(MlpTrainTcParams));
          memcpy(&M->tg_train_maps, p.kernelParams[1], sizeof(TrainStoreMaps));
        }
      }
    }
    cudaGraphExec_t ex = nullptr;
    if (adam && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
      M->tg_graph = g;  // kept: tg_adam is one of its nodes
      g = nullptr;
      M->tg_exec = ex;
      M->tg_adam = adam;
      M->tg_adam_params = ap;
      M->tg_train = train;
      M->tg_train_params = tp;
      M->tg_n = n;
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();  // a failed capture only means eager steps
}

}  // namespace

extern "C" {

crp_status crp_mlp_create(crp_context* ctx, int32_t n_in, int32_t hidden, int32_t n_hidden,
                          uint64_t seed, crp_mlp** out) {
  if (!ctx || !out || n_in < 1 || n_in > 64 || hidden < 128 || hidden % 128 != 0 ||
      hidden > 4096 || n_hidden < 1 || n_hidden > 16) {
    set_error("crp_mlp_create: need 1 <= n_in <= 64, hidden a multiple of 128 (<= 4096), "
              "1 <= n_hidden <= 16");
    return CRP_E_INVALID;
  }
  *out = nullptr;
  crp_mlp* M = new (std::nothrow) crp_mlp;
  if (!M) {
    set_error("crp_mlp_create: host allocation failed");
    return CRP_E_OOM;
  }
  M->n_in = n_in;
  M->hidden = hidden;
  M->n_hidden = n_hidden;
  M->n_out = 3;
  M->step = 0;
  M->cap = 0;
  M->dz = M->dz2 = M->dzt = M->ht = nullptr;
  M->y = M->dy = M->loss = nullptr;
  M->tcap = 0;
  M->dzT = M->dzT2 = M->dzT3 = nullptr;
  M->use_graph = true;
  M->tg_graph = nullptr;
  M->tg_exec = nullptr;
  M->tg_adam = nullptr;
  memset(&M->tg_adam_params, 0, sizeof(M->tg_adam_params));
  M->tg_train = nullptr;
  memset(&M->tg_train_params, 0, sizeof(M->tg_train_params));
  memset(&M->tg_train_args, 0, sizeof(M->tg_train_args));
  memset(&M->tg_train_maps, 0, sizeof(M->tg_train_maps));
  M->tg_n = 0;
  M->tg_stream = nullptr;
  M->xs = M->ts = nullptr;
  M->scap = 0;
  M->tc_err = nullptr;
  M->forward_path = CRP_MLP_PATH_AUTO;
  M->sm_count = 0;
  {
    DevState unused;
    uint64_t n_unused = 0, seed_unused = 0;
    context_pool(ctx, &unused, &n_unused, &M->device, &seed_unused);
    cudaSetDevice(M->device);
  }
  int64_t off = 0;
  std::vector<int64_t> offs;
  std::vector<int> fan, kind;
  for (int l = 0; l <= n_hidden; ++l) {
    const int fi = l == 0 ? n_in : hidden;
    const int fo = l == n_hidden ? 3 : hidden;
    M->w_off.push_back(off);
    offs.push_back(off);
    fan.push_back(fi);
    kind.push_back(0);
    off += (int64_t)fo * fi;
    M->b_off.push_back(off);
    offs.push_back(off);
    fan.push_back(fi);
    kind.push_back(1);
    off += fo;
  }
  M->n_params = off;
  M->params = static_cast<float*>(dev_alloc(sizeof(float) * off));
  M->grad = static_cast<float*>(dev_alloc(sizeof(float) * off));
  M->m = static_cast<float*>(dev_alloc(sizeof(float) * off));
  M->v = static_cast<float*>(dev_alloc(sizeof(float) * off));
  M->wb.assign(n_hidden, nullptr);
  M->wbt.assign(n_hidden, nullptr);
  bool ok = M->params && M->grad && M->m && M->v;
  M->forward_path = CRP_MLP_PATH_AUTO;
  cudaDeviceGetAttribute(&M->sm_count, cudaDevAttrMultiProcessorCount, M->device);
  const bool tc = mlp_tc_supported(n_in, hidden, n_hidden, 3);
  if (tc) {
    M->wimg.assign(n_hidden, nullptr);
    M->wimgT.assign(n_hidden, nullptr);
    M->tc_err = static_cast<unsigned*>(dev_alloc(sizeof(unsigned)));
    ok = ok && M->tc_err;
    if (M->tc_err) cudaMemset(M->tc_err, 0, sizeof(unsigned));
  }
  for (int l = 1; l < n_hidden; ++l) {
    M->wb[l] = static_cast<__nv_bfloat16*>(dev_alloc(sizeof(__nv_bfloat16) * hidden * hidden));
    M->wbt[l] = static_cast<__nv_bfloat16*>(dev_alloc(sizeof(__nv_bfloat16) * hidden * hidden));
    ok = ok && M->wb[l] && M->wbt[l];
    if (tc) {
      M->wimg[l] = static_cast<__nv_bfloat16*>(dev_alloc(sizeof(__nv_bfloat16) * hidden * hidden));
      M->wimgT[l] = static_cast<__nv_bfloat16*>(dev_alloc(sizeof(__nv_bfloat16) * hidden * hidden));
      ok = ok && M->wimg[l] && M->wimgT[l];
    }
  }
  int64_t* d_off = static_cast<int64_t*>(dev_alloc(sizeof(int64_t) * offs.size()));
  int* d_fan = static_cast<int*>(dev_alloc(sizeof(int) * fan.size()));
  int* d_kind = static_cast<int*>(dev_alloc(sizeof(int) * kind.size()));
  crp_status st = CRP_OK;
  if (!ok || !d_off || !d_fan || !d_kind) {
    st = CRP_E_OOM;
    set_error("crp_mlp_create: device allocation failed");
  } else {
    cudaMemcpy(d_off, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d_fan, fan.data(), sizeof(int) * fan.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d_kind, kind.data(), sizeof(int) * kind.size(), cudaMemcpyHostToDevice);
    k_init<<<nblk(off, 256), 256>>>(M->params, off, d_off, d_fan, d_kind, n_hidden + 1, seed);
    cudaMemset(M->m, 0, sizeof(float) * off);
    cudaMemset(M->v, 0, sizeof(float) * off);
    st = refresh_bf16(M, 0);
    const cudaError_t e = cudaDeviceSynchronize();
    if (st == CRP_OK && e != cudaSuccess) st = fail_cuda(e, "crp_mlp_create");
  }
  dev_free(d_off);
  dev_free(d_fan);
  dev_free(d_kind);
  if (st != CRP_OK) {
    crp_mlp_destroy(M);
    return st;
  }
  *out = M;
  return CRP_OK;
}

crp_status crp_mlp_destroy(crp_mlp* M) {
  if (!M) return CRP_OK;
  cudaDeviceSynchronize();
  drop_graph(M);
  if (M->tg_stream) cudaStreamDestroy(M->tg_stream);
  dev_free(M->xs);
  dev_free(M->ts);
  free_ws(M);
  free_tws(M);
  dev_free(M->params);
  dev_free(M->grad);
  dev_free(M->m);
  dev_free(M->v);
  for (auto* p : M->wb) dev_free(p);
  for (auto* p : M->wbt) dev_free(p);
  for (auto* p : M->wimg) dev_free(p);
  for (auto* p : M->wimgT) dev_free(p);
  dev_free(M->tc_err);
  delete M;
  return CRP_OK;
}

int64_t crp_mlp_num_params(const crp_mlp* M) { return M ? M->n_params : 0; }

crp_status crp_mlp_set_params(crp_mlp* M, const float* host) {
  if (!M || !host) {
    set_error("crp_mlp_set_params: NULL argument");
    return CRP_E_INVALID;
  }
  cudaError_t e = cudaMemcpy(M->params, host, sizeof(float) * M->n_params, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_cuda(e, "crp_mlp_set_params");
  cudaMemset(M->m, 0, sizeof(float) * M->n_params);
  cudaMemset(M->v, 0, sizeof(float) * M->n_params);
  M->step = 0;
  crp_status st = refresh_bf16(M, 0);
  e = cudaDeviceSynchronize();
  return st != CRP_OK ? st : (e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_mlp_set_params"));
}

crp_status crp_mlp_get_params(const crp_mlp* M, float* host, float* host_grad) {
  if (!M || (!host && !host_grad)) {
    set_error("crp_mlp_get_params: NULL argument");
    return CRP_E_INVALID;
  }
  cudaError_t e = cudaSuccess;
  if (host) e = cudaMemcpy(host, M->params, sizeof(float) * M->n_params, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && host_grad)
    e = cudaMemcpy(host_grad, M->grad, sizeof(float) * M->n_params, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_mlp_get_params");
}

crp_status crp_mlp_forward(crp_mlp* M, const float* x, float* y_hat, int64_t n, void* stream) {
  if (!M || n < 0 || (n > 0 && (!x || !y_hat))) {
    set_error("crp_mlp_forward: bad argument");
    return CRP_E_INVALID;
  }
  if (n == 0) return CRP_OK;
  if (n % 128 != 0) {
    set_error("crp_mlp_forward: n must be a multiple of 128 (got %lld)", (long long)n);
    return CRP_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tc_ok = !M->wimg.empty();
  if (M->forward_path == CRP_MLP_PATH_TENSOR_CORE_FUSED && !tc_ok) {
    set_error("crp_mlp_forward: the fused tensor-core path needs hidden = 256, n_in <= 8");
    return CRP_E_INVALID;
  }
  if (tc_ok && M->forward_path != CRP_MLP_PATH_LAYERED) {
    MlpTcParams P;
    memset(&P, 0, sizeof(P));
    P.x = x;
    P.n_in = M->n_in;
    P.n_gemm = M->n_hidden - 1;
    P.n_tiles = n / 128;
    P.W1 = M->params + M->w_off[0];
    P.b1 = M->params + M->b_off[0];
    for (int l = 1; l < M->n_hidden; ++l) {
      P.Wimg[l - 1] = M->wimg[l];
      P.bh[l - 1] = M->params + M->b_off[l];
    }
    P.Wout = M->params + M->w_off[M->n_hidden];
    P.bout = M->params + M->b_off[M->n_hidden];
    P.y = y_hat;
    P.err = M->tc_err;
    cudaError_t e = mlp_forward_tc(P, M->sm_count, s);
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, M->tc_err, sizeof(unsigned),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_mlp_forward: tensor-core forward");
    if (err) {
      cudaMemsetAsync(M->tc_err, 0, sizeof(unsigned), s);
      set_error("crp_mlp_forward: a tensor-core completion wait timed out");
      return CRP_E_CUDA;
    }
    return CRP_OK;
  }
  const int64_t chunk = n < (1 << 20) ? n : (1 << 20);  // bounds the activation workspace
  crp_status st = ensure_ws(M, chunk);
  for (int64_t r0 = 0; st == CRP_OK && r0 < n; r0 += chunk) {
    const int64_t m = n - r0 < chunk ? n - r0 : chunk;
    st = forward(M, x + r0 * M->n_in, m, nullptr, y_hat + r0 * 3, s);
  }
  return st;
}

crp_status crp_mlp_set_forward_path(crp_mlp* M, int32_t path) {
  if (!M || path < CRP_MLP_PATH_AUTO || path > CRP_MLP_PATH_LAYERED) {
    set_error("crp_mlp_set_forward_path: bad argument");
    return CRP_E_INVALID;
  }
  if (path == CRP_MLP_PATH_TENSOR_CORE_FUSED && M->wimg.empty()) {
    set_error("crp_mlp_set_forward_path: the fused tensor-core path needs hidden = 256, n_in <= 8");
    return CRP_E_INVALID;
  }
  M->forward_path = path;
  return CRP_OK;
}

crp_status crp_mlp_set_train_graph(crp_mlp* M, int32_t enable) {
  if (!M) {
    set_error("crp_mlp_set_train_graph: NULL argument");
    return CRP_E_INVALID;
  }
  M->use_graph = enable != 0;
  if (!M->use_graph) drop_graph(M);
  return CRP_OK;
}

crp_status crp_mlp_train_step(crp_mlp* M, const float* x, const float* t, int64_t n, float lr,
                              float* loss_out, void* stream) {
  if (!M || !x || !t || n < 128 || n % 128 != 0 || !(lr >= 0.f)) {
    set_error("crp_mlp_train_step: need a batch n >= 128, multiple of 128, lr >= 0");
    return CRP_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the tensor-core GEMMs whenever the fused forward is available and the
  // layered path is not forced
  const bool tc = !M->wimg.empty() && M->forward_path != CRP_MLP_PATH_LAYERED;
  crp_status st = ensure_ws(M, n);
  if (st == CRP_OK && tc) st = ensure_tws(M, n);
  // graph replay: tensor-core path, an Adam step, a stream not being captured
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  const bool graph = tc && lr > 0.f && M->use_graph && cs == cudaStreamCaptureStatusNone;
  if (st == CRP_OK && graph) st = ensure_stage(M, n);
  if (st != CRP_OK) return st;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  if (graph && M->tg_exec && M->tg_n == n) {
    cudaError_t e = cudaSuccess;
    MlpTrainTcParams tpar = M->tg_train_args;
    if (M->tg_train) {
      // the one-kernel step reads this step's x and t where they are
      tpar.x = x;
      tpar.t = t;
      void* targs[] = {&tpar, &M->tg_train_maps};
      cudaKernelNodeParams kp = M->tg_train_params;
      kp.kernelParams = targs;
      kp.extra = nullptr;
      e = cudaGraphExecKernelNodeSetParams(M->tg_exec, M->tg_train, &kp);
    } else {
      e = cudaMemcpyAsync(M->xs, x, sizeof(float) * (size_t)n * M->n_in, cudaMemcpyDeviceToDevice,
                          s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(M->ts, t, sizeof(float) * (size_t)n * 3, cudaMemcpyDeviceToDevice, s);
    }
    M->step += 1;
    float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
    float lr_ = lr;
    int64_t np = M->n_params;
    Bf16Jobs jobs;
    int nj = bf16_jobs(M, &jobs), hn = M->hidden;
    void* args[] = {&M->params, &M->grad, &M->m, &M->v, &np, &lr_, (void*)&b1, (void*)&b2,
                    (void*)&eps, &c1, &c2, &jobs, &nj, &hn};
    cudaKernelNodeParams kp = M->tg_adam_params;
    kp.kernelParams = args;
    kp.extra = nullptr;
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(M->tg_exec, M->tg_adam, &kp);
    if (e == cudaSuccess) e = cudaGraphLaunch(M->tg_exec, s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_mlp_train_step: graph replay");
  } else {
    st = step_gradients(M, x, t, n, s, tc);
    if (st == CRP_OK && lr > 0.f) {
      M->step += 1;
      const float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
      Bf16Jobs jobs;
      const int nj = bf16_jobs(M, &jobs);
      k_adam<<<adam_blocks(nj, M->hidden), 256, 0, s>>>(M->params, M->grad, M->m, M->v,
                                                         M->n_params, lr, b1, b2, eps, c1, c2, jobs,
                                                         nj, M->hidden);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = fail_cuda(e, "crp_mlp_train_step: Adam");
    }
    if (st == CRP_OK && graph) capture_train_graph(M, n);  // for the next calls
  }
  if (st == CRP_OK && loss_out) {
    float l = 0.f;
    unsigned err = 0;
    cudaError_t e = cudaMemcpyAsync(&l, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && tc)
      e = cudaMemcpyAsync(&err, M->tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_mlp_train_step");
    if (err) {
      cudaMemsetAsync(M->tc_err, 0, sizeof(unsigned), s);
      set_error("crp_mlp_train_step: a tensor-core completion wait timed out");
      return CRP_E_CUDA;
    }
    *loss_out = l / (float)n;
  }
  return st;
}

}  // extern "C"
