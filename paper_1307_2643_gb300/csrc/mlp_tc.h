// mlp_tc.h -- tensor-core (tcgen05) kernels of the MLP surrogate: the fused
// forward pass and the GEMMs of the training step.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace crp {

constexpr int kMlpTcMaxGemm = 8;

struct MlpTcParams {
  const float* x;  // [n][n_in]
  int n_in;
  int n_gemm;       // hidden-to-hidden layers (n_hidden - 1)
  int64_t n_tiles;  // n / 128
  const float* W1;  // [256][n_in]
  const float* b1;
  // hidden layer weights as bf16 tensor-core images (128-byte-swizzled
  // K-major): element (o, i) of W at (i / 64) * 16384 + o * 64 +
  // (((i / 8) % 8) ^ (o % 8)) * 8 + i % 8
  const __nv_bfloat16* Wimg[kMlpTcMaxGemm];
  const float* bh[kMlpTcMaxGemm];
  const float* Wout;  // [3][256]
  const float* bout;
  float* y;       // [n][3], unit vectors
  unsigned* err;  // set to 1 when a tensor-core wait timed out
  // training forward (mlp_forward_tc_train): the hidden activations h[l]
  // ([n][256] bf16, l = 0 the input layer's, l = k + 1 hidden GEMM k's) and
  // their transposes hT[l] ([256][ldt] bf16, null where not needed); no
  // output layer
  __nv_bfloat16* h[kMlpTcMaxGemm + 1];
  __nv_bfloat16* hT[kMlpTcMaxGemm + 1];
  int64_t ldt;
};

// Tensor-core GEMM of the training step (tcgen05, FP32 accumulation in TMEM):
// C[M][256] = A[M][K] B[256][K]^T with bf16 operands stored row-major (K
// contiguous).  Work items are 128-row tiles of C times `splits` ranges of K;
// each item's K range runs through 256-wide chunks.  Epilogues:
//   GEMM_TC_BIAS_RELU  out = bf16(max(C + bias, 0))
//   GEMM_TC_MASK       out = bf16(C where mask > 0, else 0)
//   GEMM_TC_ATOMIC     out_f += C (vector reductions; split-K partial sums)
// The first two also write out_t = out^T ([256][ldot]) when out_t is given;
// with rowsum, the row sums of A are added to it (the bias gradient when A is
// a transposed backward signal).
enum GemmTcEpi { GEMM_TC_BIAS_RELU = 0, GEMM_TC_MASK = 1, GEMM_TC_ATOMIC = 2 };
struct GemmTcParams {
  const __nv_bfloat16* A;
  int64_t lda;
  const __nv_bfloat16* B;
  int64_t ldb;
  int64_t M, K;  // M a multiple of 128, K a multiple of 16
  int splits;
  const float* bias;
  const __nv_bfloat16* mask;
  int64_t ldm;
  __nv_bfloat16* out;
  int64_t ldo;
  __nv_bfloat16* out_t;
  int64_t ldot;
  float* out_f;
  int64_t ldf;
  float* rowsum;  // optional: rowsum[m] += sum over the item's K range of A[m][k]
  // optional, GEMM_TC_MASK: the input layer's gradients from the output tile
  // (dz_0) and the inputs x [M][n_in] (n_in <= 8): gw_in[c][i] += sum_m
  // out[m][c] x[m][i], gb_in[c] += sum_m out[m][c]
  const float* xin;
  int n_in;
  float* gw_in;
  float* gb_in;
  unsigned* err;  // set to 1 when a tensor-core wait timed out
};
cudaError_t gemm_tc(int epi, const GemmTcParams& p, int device, int sm_count, cudaStream_t s);
// np (<= 3) weight-gradient problems of one shape in one launch of a
// K-pipelined kernel: out_f[256][256] += A^T B with A and B stored row-major
// [K][256] (leading dimensions lda, ldb >= 256; M = 256, the same K, a
// multiple of 64), and rowsum[m] += sum_k A[k][m].  Each work item computes a
// whole 256 x 256 output over its K range, streaming 64-row chunks through
// three shared-memory stages.
cudaError_t wgrad_tc(const GemmTcParams* ps, int np, int sm_count, cudaStream_t s);

// One training step's forward pass, output layer, loss and backward signals
// in one persistent tcgen05 kernel (hidden 256, three hidden-to-hidden
// layers): per tile of 128 samples the activations and backward signals stay
// in shared memory, the ReLU masks in registers; written out are the
// activations h_0 .. h_2 and backward signals dz_1 .. dz_3 (row-major) the
// weight-gradient GEMMs read, and the output and input layers' gradients.
constexpr int kMlpTrainGemm = 3;
struct MlpTrainTcParams {
  const float* x;  // [n][n_in]
  const float* t;  // [n][3] target unit vectors
  int n_in;
  int64_t n, n_tiles;  // n = 128 n_tiles
  const float* W1;     // [256][n_in]
  const float* b1;
  // forward images of the hidden weights W_{k+1} (as MlpTcParams::Wimg) and
  // the same images of their transposes: element (o, i) of W at
  // (o / 64) * 16384 + i * 64 + (((o / 8) % 8) ^ (i % 8)) * 8 + o % 8
  const __nv_bfloat16* Wimg[kMlpTrainGemm];
  const __nv_bfloat16* WimgT[kMlpTrainGemm];
  const float* bh[kMlpTrainGemm];
  const float* Wout;  // [3][256]
  const float* bout;
  __nv_bfloat16* h[kMlpTrainGemm];        // h_0 .. h_2, row-major [n][256]
  __nv_bfloat16* dz[kMlpTrainGemm + 1];   // dz_1 .. dz_3, row-major [n][256] (index = layer)
  float* loss;   // += sum over the batch of 1 - y_hat . t
  float* gW1;    // [256][n_in] +=
  float* gb1;    // [256] +=
  float* gWout;  // [3][256] +=
  float* gbout;  // [3] +=
  unsigned* err;  // set to 1 when a tensor-core wait timed out
};
cudaError_t mlp_train_tc(const MlpTrainTcParams& p, int sm_count, cudaStream_t s);
// The kernel's second argument: tensor maps of the row-major [n][256] outputs
// h_0 .. h_2 and dz_1 .. dz_3 (boxes of 64 columns x 128 rows, 128-byte
// swizzle) in the order of the GEMMs that read them (store s holds the input
// of GEMM s).  A captured launch has the arguments (MlpTrainTcParams,
// TrainStoreMaps); the kernel's address identifies its graph node.
struct TrainStoreMaps {
  CUtensorMap out[2 * kMlpTrainGemm];
};
const void* mlp_train_tc_kernel(int n_in);

// Element count of one hidden layer's weight image (256 x 256).
size_t mlp_tc_weight_image_elems();
bool mlp_tc_supported(int n_in, int hidden, int n_hidden, int n_out);
cudaError_t mlp_forward_tc(const MlpTcParams& p, int sm_count, cudaStream_t s);
// The forward pass of a training step on the same kernel: stores every hidden
// activation (and the transposes p.hT asks for) instead of the output layer.
cudaError_t mlp_forward_tc_train(const MlpTcParams& p, int sm_count, cudaStream_t s);

}  // namespace crp
