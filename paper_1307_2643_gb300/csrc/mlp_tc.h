// mlp_tc.h -- fused tensor-core (tcgen05) forward pass of the MLP surrogate.
#pragma once

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
  // hidden layer weights as bf16 core-matrix images: element (o, i) of W at
  // (o / 8) * 2048 + (i / 8) * 64 + (o % 8) * 8 + i % 8
  const __nv_bfloat16* Wimg[kMlpTcMaxGemm];
  const float* bh[kMlpTcMaxGemm];
  const float* Wout;  // [3][256]
  const float* bout;
  float* y;       // [n][3], unit vectors
  unsigned* err;  // set to 1 when a tensor-core wait timed out
};

// Element count of one hidden layer's weight image (256 x 256).
size_t mlp_tc_weight_image_elems();
bool mlp_tc_supported(int n_in, int hidden, int n_hidden, int n_out);
cudaError_t mlp_forward_tc(const MlpTcParams& p, int sm_count, cudaStream_t s);

}  // namespace crp
