// mlp_tc.cu -- fused forward pass of the MLP lens surrogate on the
// fifth-generation tensor cores (tcgen05, TMEM accumulators).
//
// One CTA (two warpgroups, 256 threads) per tile of 128 samples, persistent
// over tiles; thread t owns row t % 128 and, in the CUDA-core phases, the
// columns of half t / 128.  The activations of a tile never leave the SM:
//   * input layer (K = n_in, FP32 on the CUDA cores) -> bf16 tile A in shared
//     memory (128 x 256, K-major core-matrix layout, 64 KB);
//   * each hidden 256 -> 256 layer: its bf16 weights (stored in global memory
//     as a 128 KB image in the 128-byte-swizzled K-major layout: four
//     64-column blocks of 256 rows x 128 bytes, a row's 16-byte chunks XOR-ed
//     with the row index mod 8) are copied into shared tile B by one bulk
//     copy; one thread issues 16 tcgen05.mma (M 128, N 256, K 16,
//     bf16 x bf16 -> FP32) into 256 TMEM columns and commits them to an
//     mbarrier; every warp then reads its 32 TMEM lanes (rows) with
//     tcgen05.ld, adds the bias, applies ReLU and writes the bf16 result back
//     into tile A as the next layer's operand;
//   * the last hidden layer's epilogue feeds the thin output layer (N = 3,
//     FP32) and the normalisation directly.
// Tile A's layout here (no swizzle, K-major): 8 x 8 bf16 core
// matrices of 128 contiguous bytes (row r of the core matrix at 16 r); the
// core matrix of rows 8g.. and columns 8j.. sits at g * SBO + j * LBO with
// LBO = 128 B (next 8 columns, the K direction) and SBO = 4096 B (next 8
// rows): row-group-major, so element (r, k) is at
// (r / 8) * 4096 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "crp_internal.cuh"
#include "mlp_tc.h"

namespace crp {
namespace {

constexpr int kRows = 128;     // samples per tile (MMA M)
constexpr int kH = 256;        // hidden width (MMA N and total K)
constexpr int kThreads = 256;  // two warpgroups; warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kMaxIn = 8;
constexpr uint32_t kABytes = kRows * kH * 2;
constexpr uint32_t kBBytes = kH * kH * 2;
constexpr uint32_t kBBlock = kH * 128;     // tile B: 64-column blocks of 256 rows x 128 B
constexpr uint32_t kLbo = 128;             // next 8-column (K) group
constexpr uint32_t kSbo = (kH / 8) * 128;  // next 8-row group: 4096
constexpr uint32_t kTmemCols = 256;
// small parameters staged once per CTA: W1 (padded to 8 inputs), b1, hidden
// biases, W_out, b_out, and the second warpgroup's output-layer partial sums
constexpr size_t kParFloats = kH * kMaxIn + kH + kMlpTcMaxGemm * kH + 3 * kH + 4 + 3 * kRows;
constexpr size_t kSmem = 1024 + kABytes + kBBytes + 64 + kParFloats * 4;
constexpr long long kSpinLimit = 1ll << 22;

// tcgen05 instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B
// bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading- and stride-
// dimension byte offsets (all >> 4, 14 bits each), descriptor version 1
// (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Descriptor of a 128-byte-swizzled K-major operand: start address, leading
// byte offset 16 (unused within a swizzle atom), 1024 bytes between groups
// of 8 rows, version 1, swizzle mode 2 (128 B) in bits 61-63.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Bounded wait for the mbarrier phase with the given parity.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// bf16 pair of max(lo, 0), max(hi, 0), rounded to nearest even (low half lo).
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Store row `row`'s bf16 values of columns c0 .. c0 + 8 q - 1 (packed pairs w)
// into h (row-major, ld 256: q 16-byte stores) and, when hT is given, into the
// transpose (ld ldt: one 2-byte store per column; a warp's 32 consecutive rows
// make each column's stores one contiguous 64-byte run).
template <int Q>
__device__ __forceinline__ void store_activation(const uint32_t* w, int64_t row, int c0,
                                                 __nv_bfloat16* h, __nv_bfloat16* hT,
                                                 int64_t ldt) {
  uint4* dst = reinterpret_cast<uint4*>(h + row * kH + c0);
#pragma unroll
  for (int q = 0; q < Q; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
  if (hT) {
    unsigned short* t = reinterpret_cast<unsigned short*>(hT);
#pragma unroll
    for (int j = 0; j < 8 * Q; ++j)
      t[(int64_t)(c0 + j) * ldt + row] = (unsigned short)(w[j / 2] >> (16 * (j & 1)));
  }
}

// NIN: compiled input count (4 for the surrogate's inputs); 0 = any n_in <= 8
// (weights zero-padded to 8 inputs).  TRAIN: the forward pass of a training
// step -- every hidden activation stored (store_activation), no output layer.
template <int NIN, bool TRAIN>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_forward_tc(const MlpTcParams P) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* base = tc_smem + ((1024u - (smem_u32(tc_smem) & 1023u)) & 1023u);
  unsigned char* As = base;
  unsigned char* Bs = base + kABytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + kBBytes);  // MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  uint64_t* wbar = bar + 2;  // weight image landed in tile B
  float* sW1 = reinterpret_cast<float*>(Bs + kBBytes + 64);  // [kH][kMaxIn]
  float* sb1 = sW1 + kH * kMaxIn;
  float* sbh = sb1 + kH;                       // [kMlpTcMaxGemm][kH]
  float* sWo = sbh + kMlpTcMaxGemm * kH;       // [3][kH]
  float* sbo = sWo + 3 * kH;                   // [4]
  float* sy = sbo + 4;                         // [3][kRows]
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & (kRows - 1);  // row of the tile this thread owns
  const int g = tid >> 7;           // warpgroup: columns [128 g, 128 g + 128)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(wbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int e = tid; e < kH * kMaxIn; e += kThreads) {
    const int o = e / kMaxIn, i = e % kMaxIn;
    sW1[e] = i < P.n_in ? P.W1[o * P.n_in + i] : 0.f;
  }
  for (int e = tid; e < kH; e += kThreads) sb1[e] = P.b1[e];
  for (int l = 0; l < P.n_gemm; ++l)
    for (int e = tid; e < kH; e += kThreads) sbh[l * kH + e] = P.bh[l][e];
  for (int e = tid; e < 3 * kH; e += kThreads) sWo[e] = P.Wout[e];
  if (tid < 3) sbo[tid] = P.bout[tid];
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_warp = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t parity = 0, wparity = 0;
  bool failed = false, wpend = false;
  // weights of the first layer for the first tile; later copies are issued as
  // soon as the previous MMAs have released tile B, so they overlap the
  // epilogue (one bulk copy, started by thread 0, tracked by every thread)
  auto fetch_weights = [&](int l) {
    if (tid == 0) {
      bar_expect_tx(wbar, kBBytes);
      bulk_copy_g2s(Bs, P.Wimg[l], kBBytes, wbar);
    }
    wpend = true;
  };
  if (blockIdx.x < P.n_tiles) fetch_weights(0);

  for (int64_t tile = blockIdx.x; tile < P.n_tiles && !failed; tile += gridDim.x) {
    const int64_t row = tile * kRows + r;
    // ---- input layer (FP32): this warpgroup's 128 outputs of row r ----
    constexpr int NI = NIN > 0 ? NIN : kMaxIn;  // inputs summed (zero-padded when NIN = 0)
    float xin[kMaxIn];
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i)
      xin[i] = (NIN > 0 ? i < NIN : i < P.n_in) ? P.x[row * (NIN > 0 ? NIN : P.n_in) + i] : 0.f;
#pragma unroll 2
    for (int kc = 16 * g; kc < 16 * g + 16; ++kc) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 8; e += 4) {
        const float4 bb = *reinterpret_cast<const float4*>(sb1 + kc * 8 + e);
        const float bq[4] = {bb.x, bb.y, bb.z, bb.w};
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = kc * 8 + e + q;
          const float4* wr = reinterpret_cast<const float4*>(sW1 + o * kMaxIn);
          const float4 w0 = wr[0];
          float acc = bq[q];
          acc = fmaf(w0.x, xin[0], acc);
          if (NI > 1) acc = fmaf(w0.y, xin[1], acc);
          if (NI > 2) acc = fmaf(w0.z, xin[2], acc);
          if (NI > 3) acc = fmaf(w0.w, xin[3], acc);
          if (NI > 4) {
            const float4 w1 = wr[1];
            acc = fmaf(w1.x, xin[4], acc);
            if (NI > 5) acc = fmaf(w1.y, xin[5], acc);
            if (NI > 6) acc = fmaf(w1.z, xin[6], acc);
            if (NI > 7) acc = fmaf(w1.w, xin[7], acc);
          }
          v[q] = acc;
        }
        w[e / 2] = pack_bf16_relu(v[0], v[1]);
        w[e / 2 + 1] = pack_bf16_relu(v[2], v[3]);
      }
      if (TRAIN) store_activation<1>(w, row, kc * 8, P.h[0], P.hT[0], P.ldt);
      *reinterpret_cast<uint4*>(As + (r >> 3) * kSbo + kc * kLbo + (r & 7) * 16) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
    // ---- hidden layers on the tensor cores ----
    for (int l = 0; l < P.n_gemm; ++l) {
      // generic-proxy writes of A -> visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      bool wok = bar_wait(wbar, wparity);  // this layer's weights are in B
      if (!wok) wok = bar_wait(wbar, wparity);
      if (wok) {
        wparity ^= 1u;
        wpend = false;
      }
      if (tid == 0 && wok) {
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll 1
        for (int k = 0; k < kH / 16; ++k)
          mma_bf16(tmem, sdesc(a0 + 2u * k * kLbo, kLbo, kSbo),
                   sdesc_sw128(b0 + (uint32_t)(k >> 2) * kBBlock + 32u * (uint32_t)(k & 3)), kIdesc,
                   k > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      bool ok = wok && bar_wait(bar, parity);
      if (wok && !ok) ok = bar_wait(bar, parity);  // a second bounded wait before giving up
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(P.err, 1u);
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // the MMAs are complete: tile B is free for the next weights
      if (l + 1 < P.n_gemm)
        fetch_weights(l + 1);
      else if (tile + gridDim.x < P.n_tiles)
        fetch_weights(0);
      const float* bias = sbh + l * kH;
      const bool last = l == P.n_gemm - 1;
      float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll 1
      for (int cc = 4 * g; cc < 4 * g + 4; ++cc) {
        uint32_t v[32];
        tmem_ld32(tmem_warp + (uint32_t)(cc * 32), v);
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const int col = cc * 32 + j;
          const float4 b4 = *reinterpret_cast<const float4*>(bias + col);
          w[j / 2] = pack_bf16_relu(__uint_as_float(v[j]) + b4.x, __uint_as_float(v[j + 1]) + b4.y);
          w[j / 2 + 1] =
              pack_bf16_relu(__uint_as_float(v[j + 2]) + b4.z, __uint_as_float(v[j + 3]) + b4.w);
          if (last && !TRAIN) {
            const __nv_bfloat162 p01 = *reinterpret_cast<const __nv_bfloat162*>(&w[j / 2]);
            const __nv_bfloat162 p23 = *reinterpret_cast<const __nv_bfloat162*>(&w[j / 2 + 1]);
            const float a0 = __low2float(p01), a1 = __high2float(p01);
            const float a2 = __low2float(p23), a3 = __high2float(p23);
            const float4 wa = *reinterpret_cast<const float4*>(sWo + col);
            const float4 wb = *reinterpret_cast<const float4*>(sWo + kH + col);
            const float4 wc = *reinterpret_cast<const float4*>(sWo + 2 * kH + col);
            y0 = fmaf(wa.x, a0, y0);
            y0 = fmaf(wa.y, a1, y0);
            y0 = fmaf(wa.z, a2, y0);
            y0 = fmaf(wa.w, a3, y0);
            y1 = fmaf(wb.x, a0, y1);
            y1 = fmaf(wb.y, a1, y1);
            y1 = fmaf(wb.z, a2, y1);
            y1 = fmaf(wb.w, a3, y1);
            y2 = fmaf(wc.x, a0, y2);
            y2 = fmaf(wc.y, a1, y2);
            y2 = fmaf(wc.z, a2, y2);
            y2 = fmaf(wc.w, a3, y2);
          }
        }
        if (TRAIN) store_activation<4>(w, row, cc * 32, P.h[l + 1], P.hT[l + 1], P.ldt);
        if (!last) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(As + (r >> 3) * kSbo + (cc * 4 + q) * kLbo + (r & 7) * 16) =
                make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
      }
      if (last && g == 1 && !TRAIN) {
        sy[r] = y0;
        sy[kRows + r] = y1;
        sy[2 * kRows + r] = y2;
      }
      // TMEM reads done, A rewritten and partial sums posted before moving on
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (last && g == 0 && !TRAIN) {
        y0 += sy[r] + sbo[0];
        y1 += sy[kRows + r] + sbo[1];
        y2 += sy[2 * kRows + r] + sbo[2];
        const float nrm = sqrtf(y0 * y0 + y1 * y1 + y2 * y2);
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        P.y[row * 3] = y0 * inv;
        P.y[row * 3 + 1] = y1 * inv;
        P.y[row * 3 + 2] = y2 * inv;
      }
    }
  }
  // a timed-out MMA wait: one more bounded wait for those MMAs before the
  // TMEM is given up (the phase that did not complete has parity ^ 1)
  if (failed && tid == 0) {
    bar_wait(bar, parity ^ 1u);
    if (wpend) bar_wait(wbar, wparity);  // a weight copy still in flight
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}




// One 2D TMA box (64 columns x the map's box rows) at column x, row y.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Store / add one 2D box from shared memory to global through the TMA (bulk
// async group of the issuing thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, int x, int y,
                                                  const void* src) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], "
      "[%3];\n" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// A whole training step's per-sample work in one kernel (hidden 256, three
// hidden-to-hidden layers), with the forward kernel's layout and thread roles.
// Per tile of 128 samples:
//   * input layer -> h_0 (tile A); GEMMs with W_1 .. W_3 -> h_1 .. h_3 (bias,
//     ReLU); h_0 .. h_2 also written out (row-major) for the weight
//     gradients, and their ReLU masks kept as bits in registers (thread
//     (row r, half g): word q covers columns 128 g + 32 q + [0, 32), bit e
//     the column 2 e, bit 16 + e the column 2 e + 1);
//   * output layer on the CUDA cores: y = W_out h_3 + b_out from the two
//     warpgroups' partial sums, y_hat = y / |y|, the loss term 1 - y_hat . t
//     and dy = -(t - (y_hat . t) y_hat) / |y| / n; per column c the output
//     layer's gradients sum_r dy[r] h_3[r][c] (tensor cores: tile A read as
//     the MN-major operand against dy's high and low bf16 parts in tile S);
//     then dz_3 = bf16((dy . W_out[:, c]) where h_3 > 0), one MMA of K 16 (the
//     parts of dy against those of W_out), in place in tile A;
//   * GEMMs with W_3^T, W_2^T, W_1^T (images of the transposed weights) ->
//     dz_2, dz_1, dz_0 = bf16(C where h_{l-1} > 0) in tile A (dz_3 .. dz_1 also
//     written out, row-major, for the weight gradients);
//   * per column c the input layer's gradients sum_r dz_0[r][c] x[r][i] and
//     sum_r dz_0[r][c] (tensor cores: tile A against x's parts and a ones
//     row in tile S).
// The six weight images of a tile are copied into tile B in that order (one
// bulk copy each, completing on an mbarrier), each as soon as the previous
// GEMM's MMAs have completed; each GEMM's input in tile A is written out by
// TMA while its MMAs run.  Gradient partial sums
// stay in registers over the CTA's tiles and are added to global memory once.
// The values are rounded to bf16 where the layered training step rounds them
// (activations, backward signals), so the two give the same step up to the
// order of FP32 summation and the 2^-16 relative error of the high and low
// parts (products of bf16 values are exact in FP32).
// ---------------------------------------------------------------------------
// The column tile S of the training kernel: 32 rows (n) x 128 columns (the
// tile's rows r) of bf16, 128-byte-swizzled K-major (two 64-column blocks of
// 32 rows x 128 bytes): rows 0..2 / 3..5 the high / low bf16 parts of dy,
// rows 9..11 the high parts again, row 8 ones, rows 6, 7, 12..15 zero, rows
// 16..23 / 24..31 the high / low parts of the inputs x.
constexpr uint32_t kSBytes = 32 * kRows * 2;
// Region U (8 KB): the output layer's partial sums (FP32 [2][3][kRows]), then,
// once they are read, the W_out tile: [256 c][16 k] bf16, K-major without
// swizzle (8 x 8 core matrices: LBO 128 B next 8 k, SBO 256 B next 8 c),
// k = 0..2 and 3..5 the high parts of W_out[k % 3][c], 9..11 the low parts.
constexpr uint32_t kUBytes = kH * 16 * 2;
static_assert(kUBytes >= 6 * kRows * 4, "region U holds the output-layer partial sums");
constexpr size_t kTrainFloats = kH * kMaxIn + kH + kMlpTrainGemm * kH + 3 * kH + 4 + kRows;
constexpr size_t kTrainSmem = 1024 + kABytes + kBBytes + kSBytes + kUBytes + 64 + kTrainFloats * 4;
static_assert(kTrainSmem <= 232448, "shared memory of the training kernel");
static_assert(kH == kThreads && (kH * kMaxIn) % kThreads == 0, "parameter staging of the training kernel");

// Byte offset of the 16-byte chunk q (columns 8 q .. 8 q + 7) of row r in the
// training kernel's tile A: 128 rows x 256 bf16 columns, 128-byte-swizzled
// K-major (four 64-column blocks of 16 KB; a row's 128 bytes of a block at
// 128 r, its chunks XOR-ed with r % 8), the layout of a TMA box of 64 columns
// x 128 rows with the 128-byte swizzle.
__device__ __forceinline__ uint32_t sw_chunk(int r, int q) {
  return (uint32_t)((q >> 3) * 16384 + r * 128 + (((q & 7) ^ (r & 7)) << 4));
}

// Byte offset of element (n, r) in the column tile S.
__device__ __forceinline__ uint32_t s_elem(int n, int r) {
  return (uint32_t)((r >> 6) * 4096 + n * 128 + ((((r & 63) >> 3) ^ (n & 7)) << 4) + (r & 7) * 2);
}

// bf16 high and low parts of x: x ~ hi + lo to 2^-16 relative, and the
// product of either with a bf16 is exact in FP32.
__device__ __forceinline__ void split_bf16(float x, unsigned short& hi, unsigned short& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = *reinterpret_cast<const unsigned short*>(&h);
  lo = *reinterpret_cast<const unsigned short*>(&l);
}

// Descriptor of a 128-byte-swizzled MN-major operand: 64 MN-contiguous
// elements per 128-byte row, one row per K; leading byte offset `lbo` between
// 64-element MN groups, 1024 bytes between groups of 8 K rows.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t addr, uint32_t lbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// kind::f16 instruction descriptors of the column reductions: M 128, N 16 or
// 32, A MN-major (tile A read by columns), B K-major (tile S).
constexpr uint32_t kIdescCol16 =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (2u << 17) | ((uint32_t)(kRows >> 4) << 24);
constexpr uint32_t kIdescCol32 =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (4u << 17) | ((uint32_t)(kRows >> 4) << 24);
// dz_3 = dy W_out: M 128 (rows), N 256, K 16, A MN-major (tile S), B K-major
constexpr uint32_t kIdescDz = kIdesc | (1u << 15);

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// ReLU masks.  A half of a packed pair of ReLU outputs (bf16, +0, -0 or
// positive) is positive iff adding 0x7fff to it sets its bit 15 while its
// own bit 15 is clear; no such half carries into the other.  Pair e of a
// 32-column chunk (columns 2 e, 2 e + 1) is kept as bits e and 16 + e of the
// chunk's mask; pair_flags(w, e) returns them in place.
__device__ __forceinline__ uint32_t pair_flags(uint32_t w, int e) {
  return ((w + 0x7fff7fffu) & ~w & 0x80008000u) >> (15 - e);
}
// The pair's halves kept where its mask bits are set, zeroed elsewhere.
__device__ __forceinline__ uint32_t keep_pair(uint32_t p, uint32_t m, int e) {
  return p & (((m >> e) & 0x10001u) * 0xffffu);
}


// Word q of a 4-word register array without dynamic indexing.
__device__ __forceinline__ uint32_t word_of(const uint32_t (&m)[4], int q) {
  return q == 0 ? m[0] : (q == 1 ? m[1] : (q == 2 ? m[2] : m[3]));
}
__device__ __forceinline__ void set_word(uint32_t (&m)[4], int q, uint32_t v) {
  m[0] = q == 0 ? v : m[0];
  m[1] = q == 1 ? v : m[1];
  m[2] = q == 2 ? v : m[2];
  m[3] = q == 3 ? v : m[3];
}

template <int NIN>
__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_train_tc(const MlpTrainTcParams P, const __grid_constant__ TrainStoreMaps T) {
  constexpr int NG = kMlpTrainGemm;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* base = tc_smem + ((1024u - (smem_u32(tc_smem) & 1023u)) & 1023u);
  unsigned char* As = base;
  unsigned char* Bs = base + kABytes;
  unsigned char* Ss = Bs + kBBytes;   // column tile S
  unsigned char* Us = Ss + kSBytes;   // region U
  uint64_t* bar = reinterpret_cast<uint64_t*>(Us + kUBytes);  // MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  uint64_t* wbar = bar + 2;  // weight image landed in tile B
  float* sW1 = reinterpret_cast<float*>(Us + kUBytes + 64);  // [kH][kMaxIn]
  float* sb1 = sW1 + kH * kMaxIn;
  float* sbh = sb1 + kH;        // [NG][kH]
  float* sWo = sbh + NG * kH;   // [3][kH]
  float* sbo = sWo + 3 * kH;    // [4]
  float* sl = sbo + 4;  // [4 warps][4]: their sums of dy and of the loss terms
  float* sy = reinterpret_cast<float*>(Us);  // [2 halves][3][kRows] output-layer partial sums
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & (kRows - 1);  // row of the tile this thread owns
  const int g = tid >> 7;           // warpgroup: columns [128 g, 128 g + 128)
  constexpr int NI = NIN > 0 ? NIN : kMaxIn;  // inputs summed (zero-padded when NIN = 0)
  // row r's inputs of a tile, loaded one tile ahead (the first before the
  // parameters are staged)
  float xnext[kMaxIn];
  auto load_x = [&](int64_t tile) {
    const int64_t row = tile * kRows + r;
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i)
      xnext[i] = tile < P.n_tiles && (NIN > 0 ? i < NIN : i < P.n_in)
                     ? P.x[row * (NIN > 0 ? NIN : P.n_in) + i]
                     : 0.f;
  };
  load_x(blockIdx.x);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(wbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    // the first GEMM's weights, copied while the small parameters are staged
    if (blockIdx.x < P.n_tiles) {
      bar_expect_tx(wbar, kBBytes);
      bulk_copy_g2s(Bs, P.Wimg[0], kBBytes, wbar);
    }
  }
  {
    // the small parameters: every load in flight before the first store
    // (kH = kThreads: one value of each kH-vector per thread)
    constexpr int kW1 = kH * kMaxIn / kThreads;
    float w1v[kW1], bhv[NG], wov[3];
#pragma unroll
    for (int k = 0; k < kW1; ++k) {
      const int e = tid + k * kThreads, o = e / kMaxIn, i = e % kMaxIn;
      w1v[k] = i < P.n_in ? P.W1[o * P.n_in + i] : 0.f;
    }
    const float b1v = P.b1[tid];
#pragma unroll
    for (int l = 0; l < NG; ++l) bhv[l] = P.bh[l][tid];
#pragma unroll
    for (int k = 0; k < 3; ++k) wov[k] = P.Wout[tid + k * kThreads];
    const float bov = tid < 3 ? P.bout[tid] : 0.f;
#pragma unroll
    for (int k = 0; k < kW1; ++k) sW1[tid + k * kThreads] = w1v[k];
    sb1[tid] = b1v;
#pragma unroll
    for (int l = 0; l < NG; ++l) sbh[l * kH + tid] = bhv[l];
#pragma unroll
    for (int k = 0; k < 3; ++k) sWo[tid + k * kThreads] = wov[k];
    if (tid < 3) sbo[tid] = bov;
    // S's ones row (the bias gradient's column sums) and its zero rows (the
    // dz_3 product reads rows 0..15 against zero W_out columns there)
    if (tid < kRows) {
      *reinterpret_cast<unsigned short*>(Ss + s_elem(8, tid)) = 0x3F80u;
      const int zr[6] = {6, 7, 12, 13, 14, 15};
#pragma unroll
      for (int z = 0; z < 6; ++z) *reinterpret_cast<unsigned short*>(Ss + s_elem(zr[z], tid)) = 0;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_warp = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t parity = 0, wparity = 0;
  bool failed = false, wpend = blockIdx.x < P.n_tiles;  // the first copy, started above
  const float inv_n = 1.f / (float)P.n;
  // the tile's weight schedule: W_1 .. W_NG, then W_NG^T .. W_1^T (every
  // thread tracks the copy; thread 0 starts it)
  auto fetch = [&](int s) {
    if (tid == 0) {
      bar_expect_tx(wbar, kBBytes);
      bulk_copy_g2s(Bs, s < NG ? P.Wimg[s] : P.WimgT[2 * NG - 1 - s], kBBytes, wbar);
    }
    wpend = true;
  };
  // step s of the schedule on tiles A and B: wait for its weights, write
  // tile A (the GEMM's input) out by TMA, 16 MMAs, wait for their completion
  // (bounded) and for the TMA's reads of tile A, start copying the next
  // weights; false on a timed-out wait
  auto gemm_step = [&](int s, bool more_tiles, int64_t tile) -> bool {
    // generic-proxy writes of A -> visible to the tensor cores and the TMA
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    bool wok = bar_wait(wbar, wparity);  // this GEMM's weights are in tile B
    if (!wok) wok = bar_wait(wbar, wparity);
    if (wok) {
      wparity ^= 1u;
      wpend = false;
    }
    if (tid == 0 && wok) {
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      for (int b = 0; b < 4; ++b) tma_store_2d(&T.out[s], 64 * b, (int)(tile * kRows), As + b * 16384);
      bulk_commit();
#pragma unroll 1
      for (int k = 0; k < kH / 16; ++k)
        mma_bf16(tmem, sdesc_sw128(a0 + (uint32_t)(k >> 2) * 16384u + 32u * (uint32_t)(k & 3)),
                 sdesc_sw128(b0 + (uint32_t)(k >> 2) * kBBlock + 32u * (uint32_t)(k & 3)), kIdesc,
                 k > 0 ? 1u : 0u);
      mma_commit(bar);
    }
    bool ok = wok && bar_wait(bar, parity);
    if (wok && !ok) ok = bar_wait(bar, parity);  // a second bounded wait before giving up
    if (tid == 0) bulk_wait_read();  // tile A may be rewritten once the TMA has read it
    parity ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(P.err, 1u);
      return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // the MMAs are complete: tile B is free for the next weights
    if (s + 1 < 2 * NG)
      fetch(s + 1);
    else if (more_tiles)
      fetch(0);
    return true;
  };
  auto after_epilogue = [&]() {
    // TMEM reads done and tile A rewritten before the next MMAs
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  };
  // a tensor-core step on shared-memory operands already written: issue
  // (thread 0), commit, bounded wait; false on a timed-out wait
  auto tc_step = [&](auto issue) -> bool {
    // generic-proxy writes of the operands -> visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      issue();
      mma_commit(bar);
    }
    bool ok = bar_wait(bar, parity);
    if (!ok) ok = bar_wait(bar, parity);
    parity ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(P.err, 1u);
      return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return true;
  };
  // the column reduction D[c][n] = sum_r A[r][c] S[n][r] for both column
  // halves (c in [128 h, 128 h + 128) -> TMEM lanes, columns n_cols h + n):
  // 2 x 8 MMAs of K 16
  auto col_mma = [&](uint32_t idesc, uint32_t n_cols) -> bool {
    return tc_step([&] {
      const uint32_t a0 = smem_u32(As), s0 = smem_u32(Ss);
#pragma unroll 1
      for (int h = 0; h < 2; ++h)
#pragma unroll 1
        for (int k = 0; k < kRows / 16; ++k)
          mma_bf16(tmem + n_cols * (uint32_t)h, sdesc_mn(a0 + 32768u * h + 2048u * k, 16384u),
                   sdesc_sw128(s0 + (uint32_t)(k >> 2) * 4096u + 32u * (uint32_t)(k & 3)), idesc,
                   k > 0 ? 1u : 0u);
    });
  };
  // gradient partial sums over this CTA's tiles: output and input layer of
  // column tid; tid 0..2: db_out, tid 3: the loss
  float go0 = 0.f, go1 = 0.f, go2 = 0.f, gib = 0.f, gsmall = 0.f;
  float gi[kMaxIn];
#pragma unroll
  for (int i = 0; i < kMaxIn; ++i) gi[i] = 0.f;

  for (int64_t tile = blockIdx.x; tile < P.n_tiles && !failed; tile += gridDim.x) {
    const int64_t row = tile * kRows + r;
    const bool more = tile + gridDim.x < P.n_tiles;
    // the targets, first needed after the forward pass
    const float t0 = P.t[row * 3], t1 = P.t[row * 3 + 1], t2 = P.t[row * 3 + 2];
    uint32_t mk[NG][4];  // ReLU masks of h_0 .. h_{NG-1}
    // ---- input layer (FP32): this warpgroup's 128 outputs of row r ----
    float xin[kMaxIn];
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i) xin[i] = xnext[i];
    load_x(tile + gridDim.x);
    if (g == 0) {
      // the inputs' high and low parts: rows 16 + i, 24 + i of S
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        unsigned short hi, lo;
        split_bf16(xin[i], hi, lo);
        *reinterpret_cast<unsigned short*>(Ss + s_elem(16 + i, r)) = hi;
        *reinterpret_cast<unsigned short*>(Ss + s_elem(24 + i, r)) = lo;
      }
    }
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      uint32_t mq = 0;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int kc = 16 * g + 4 * q + kk;
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 8; e += 4) {
          const float4 bb = *reinterpret_cast<const float4*>(sb1 + kc * 8 + e);
          const float bq[4] = {bb.x, bb.y, bb.z, bb.w};
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = kc * 8 + e + u;
            const float4* wr = reinterpret_cast<const float4*>(sW1 + o * kMaxIn);
            const float4 w0 = wr[0];
            float acc = bq[u];
            acc = fmaf(w0.x, xin[0], acc);
            if (NI > 1) acc = fmaf(w0.y, xin[1], acc);
            if (NI > 2) acc = fmaf(w0.z, xin[2], acc);
            if (NI > 3) acc = fmaf(w0.w, xin[3], acc);
            if (NI > 4) {
              const float4 w1 = wr[1];
              acc = fmaf(w1.x, xin[4], acc);
              if (NI > 5) acc = fmaf(w1.y, xin[5], acc);
              if (NI > 6) acc = fmaf(w1.z, xin[6], acc);
              if (NI > 7) acc = fmaf(w1.w, xin[7], acc);
            }
            v[u] = acc;
          }
          w[e / 2] = pack_bf16_relu(v[0], v[1]);
          w[e / 2 + 1] = pack_bf16_relu(v[2], v[3]);
        }
        *reinterpret_cast<uint4*>(As + sw_chunk(r, kc)) = make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) mq |= pair_flags(w[i], 4 * kk + i);
      }
      set_word(mk[0], q, mq);
    }
    // ---- forward: the hidden layers on the tensor cores ----
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
    for (int j = 0; j < NG; ++j) {
      if (!gemm_step(j, more, tile)) {
        failed = true;
        break;
      }
      const float* bias = sbh + j * kH;
      const bool last = j == NG - 1;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const int cc = 4 * g + q;
        uint32_t v[32];
        tmem_ld32(tmem_warp + (uint32_t)(cc * 32), v);
        uint32_t w[16];
#pragma unroll
        for (int jj = 0; jj < 32; jj += 4) {
          const int col = cc * 32 + jj;
          const float4 b4 = *reinterpret_cast<const float4*>(bias + col);
          w[jj / 2] = pack_bf16_relu(__uint_as_float(v[jj]) + b4.x, __uint_as_float(v[jj + 1]) + b4.y);
          w[jj / 2 + 1] =
              pack_bf16_relu(__uint_as_float(v[jj + 2]) + b4.z, __uint_as_float(v[jj + 3]) + b4.w);
          if (last) {
            // the output layer reads the bf16-rounded activations
            const __nv_bfloat162 p01 = *reinterpret_cast<const __nv_bfloat162*>(&w[jj / 2]);
            const __nv_bfloat162 p23 = *reinterpret_cast<const __nv_bfloat162*>(&w[jj / 2 + 1]);
            const float a0 = __low2float(p01), a1 = __high2float(p01);
            const float a2 = __low2float(p23), a3 = __high2float(p23);
            const float4 wa = *reinterpret_cast<const float4*>(sWo + col);
            const float4 wb = *reinterpret_cast<const float4*>(sWo + kH + col);
            const float4 wc = *reinterpret_cast<const float4*>(sWo + 2 * kH + col);
            y0 = fmaf(wa.x, a0, y0);
            y0 = fmaf(wa.y, a1, y0);
            y0 = fmaf(wa.z, a2, y0);
            y0 = fmaf(wa.w, a3, y0);
            y1 = fmaf(wb.x, a0, y1);
            y1 = fmaf(wb.y, a1, y1);
            y1 = fmaf(wb.z, a2, y1);
            y1 = fmaf(wb.w, a3, y1);
            y2 = fmaf(wc.x, a0, y2);
            y2 = fmaf(wc.y, a1, y2);
            y2 = fmaf(wc.z, a2, y2);
            y2 = fmaf(wc.w, a3, y2);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          *reinterpret_cast<uint4*>(As + sw_chunk(r, cc * 4 + u)) =
              make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
        if (!last) {
          uint32_t mq = 0;
#pragma unroll
          for (int e = 0; e < 16; ++e) mq |= pair_flags(w[e], e);
          set_word(mk[j + 1], q, mq);
        }
      }
      after_epilogue();
    }
    if (failed) break;
    // ---- output layer, loss and dy (CUDA cores) ----
    sy[(3 * g) * kRows + r] = y0;
    sy[(3 * g + 1) * kRows + r] = y1;
    sy[(3 * g + 2) * kRows + r] = y2;
    __syncthreads();
    // both halves form the same y: (partial of half 0 + partial of half 1) + b
    const float Y0 = (sy[r] + sy[3 * kRows + r]) + sbo[0];
    const float Y1 = (sy[kRows + r] + sy[4 * kRows + r]) + sbo[1];
    const float Y2 = (sy[2 * kRows + r] + sy[5 * kRows + r]) + sbo[2];
    const float nrm = sqrtf(Y0 * Y0 + Y1 * Y1 + Y2 * Y2);
    const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
    const float yh0 = Y0 * inv, yh1 = Y1 * inv, yh2 = Y2 * inv;
    const float d = yh0 * t0 + yh1 * t1 + yh2 * t2;
    const float dy0 = -(t0 - d * yh0) * inv * inv_n;
    const float dy1 = -(t1 - d * yh1) * inv * inv_n;
    const float dy2 = -(t2 - d * yh2) * inv * inv_n;
    if (g == 0) {
      // dy's high and low parts: rows 0..2, 3..5 of S
      const float dyk[3] = {dy0, dy1, dy2};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        unsigned short hi, lo;
        split_bf16(dyk[k], hi, lo);
        *reinterpret_cast<unsigned short*>(Ss + s_elem(k, r)) = hi;
        *reinterpret_cast<unsigned short*>(Ss + s_elem(3 + k, r)) = lo;
        *reinterpret_cast<unsigned short*>(Ss + s_elem(9 + k, r)) = hi;
      }
      // the output biases' gradients and the loss: sums over this warp's rows
      float s0 = dy0, s1 = dy1, s2 = dy2, s3 = 1.f - d;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      }
      if ((tid & 31) == 0) {
        sl[4 * warp] = s0;
        sl[4 * warp + 1] = s1;
        sl[4 * warp + 2] = s2;
        sl[4 * warp + 3] = s3;
      }
    }
    // column tid of the output layer's weight gradients, sum_r h_3[r][c] dy[r]:
    // on the tensor cores with tile A (h_3) as the MN-major operand, the
    // parts of dy (tile S) as B; D[c][n] in TMEM columns 16 h + n
    if (!col_mma(kIdescCol16, 16)) {
      failed = true;
      break;
    }
    {
      uint32_t dv[8];
      tmem_ld8(tmem_warp + 16u * (uint32_t)g, dv);
      go0 += __uint_as_float(dv[0]) + __uint_as_float(dv[3]);
      go1 += __uint_as_float(dv[1]) + __uint_as_float(dv[4]);
      go2 += __uint_as_float(dv[2]) + __uint_as_float(dv[5]);
      if (tid < 4) gsmall += (sl[tid] + sl[4 + tid]) + (sl[8 + tid] + sl[12 + tid]);
    }
    {
      // the partial sums are read: region U becomes the W_out tile (column
      // tid: its 16 k values as two 16-byte chunks)
      uint32_t wv[8];
      unsigned short hi[3], lo[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) split_bf16(sWo[k * kH + tid], hi[k], lo[k]);
      wv[0] = hi[0] | ((uint32_t)hi[1] << 16);
      wv[1] = hi[2] | ((uint32_t)hi[0] << 16);
      wv[2] = hi[1] | ((uint32_t)hi[2] << 16);
      wv[3] = 0u;
      wv[4] = (uint32_t)lo[0] << 16;
      wv[5] = lo[1] | ((uint32_t)lo[2] << 16);
      wv[6] = 0u;
      wv[7] = 0u;
      unsigned char* wp = Us + (tid >> 3) * 256 + (tid & 7) * 16;
      *reinterpret_cast<uint4*>(wp) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      *reinterpret_cast<uint4*>(wp + 128) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    }
    // dz_3 = bf16((dy . W_out[:, c]) where h_3 > 0): one MMA of K 16 from S's
    // dy parts (MN-major A) and the W_out tile, then in place in tile A
    if (!tc_step([&] {
          mma_bf16(tmem, sdesc_mn(smem_u32(Ss), 4096u), sdesc(smem_u32(Us), 128u, 256u), kIdescDz,
                   0u);
        })) {
      failed = true;
      break;
    }
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const int cc = 4 * g + q;
      uint32_t v[32];
      tmem_ld32(tmem_warp + (uint32_t)(cc * 32), v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint4* ap = reinterpret_cast<uint4*>(As + sw_chunk(r, cc * 4 + u));
        const uint4 hq = *ap;
        const uint32_t hw[4] = {hq.x, hq.y, hq.z, hq.w};
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          w[e] = keep_pair(pack_bf16(__uint_as_float(v[8 * u + 2 * e]),
                                     __uint_as_float(v[8 * u + 2 * e + 1])),
                           pair_flags(hw[e], 0), 0);
        *ap = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    // ---- backward: dz_{l-1} = (dz_l W_l) where h_{l-1} > 0, l = NG .. 1 ----
#pragma unroll
    for (int j = NG - 1; j >= 0; --j) {
      if (!gemm_step(2 * NG - 1 - j, more, tile)) {
        failed = true;
        break;
      }
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const int cc = 4 * g + q;
        uint32_t v[32];
        tmem_ld32(tmem_warp + (uint32_t)(cc * 32), v);
        const uint32_t mw = word_of(mk[j], q);
        uint32_t w[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
          w[e] = keep_pair(pack_bf16(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1])), mw, e);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          *reinterpret_cast<uint4*>(As + sw_chunk(r, cc * 4 + u)) =
              make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
      }
      after_epilogue();
    }
    if (failed) break;
    // column tid of the input layer's gradients, sum_r dz_0[r][c] x[r][i] and
    // sum_r dz_0[r][c]: tile A (dz_0) against S's inputs and ones row
    if (!col_mma(kIdescCol32, 32)) {
      failed = true;
      break;
    }
    {
      uint32_t dv[32];
      tmem_ld32(tmem_warp + 32u * (uint32_t)g, dv);
      gib += __uint_as_float(dv[8]);
#pragma unroll
      for (int i = 0; i < NI; ++i) gi[i] += __uint_as_float(dv[16 + i]) + __uint_as_float(dv[24 + i]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // tile A and the staged inputs are rewritten by the next tile
  }
  if (!failed) {
    atomicAdd(P.gWout + tid, go0);
    atomicAdd(P.gWout + kH + tid, go1);
    atomicAdd(P.gWout + 2 * kH + tid, go2);
    constexpr int NI = NIN > 0 ? NIN : kMaxIn;
#pragma unroll
    for (int i = 0; i < NI; ++i)
      if (i < P.n_in) atomicAdd(P.gW1 + tid * P.n_in + i, gi[i]);
    atomicAdd(P.gb1 + tid, gib);
    if (tid < 3)
      atomicAdd(P.gbout + tid, gsmall);
    else if (tid == 3)
      atomicAdd(P.loss, gsmall);
  }
  // a timed-out MMA wait: one more bounded wait for those MMAs before the
  // TMEM is given up (the phase that did not complete has parity ^ 1)
  if (failed && tid == 0) {
    bar_wait(bar, parity ^ 1u);
    if (wpend) bar_wait(wbar, wparity);  // a weight copy still in flight
  }
  if (tid == 0) bulk_wait_all();  // every TMA store has completed
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Training GEMM: C[M][256] = A[M][K] B[256][K]^T on the tensor cores.
// One CTA (256 threads) per SM, persistent over work items (a 128-row tile of
// C and a range of K).  Per 256-wide K chunk one thread starts TMA copies of
// the A rows (128 x kc) and the B rows (256 x kc) in 64-column boxes into the
// 128-byte-swizzled K-major layout (rows of 128 bytes, 16-byte chunks XOR-ed
// with the row index within each 1024-byte group of 8 rows), the CTA waits
// for their bytes on an mbarrier, and the thread issues kc / 16 MMAs (M 128,
// N 256, K 16) into 256 TMEM columns; after the last chunk every thread reads
// its row's 128 accumulator columns back for the epilogue.  B stays resident
// when there is one K chunk in all (the weights of a layer); the next item's
// first chunk is copied while the epilogue runs.
// ---------------------------------------------------------------------------
constexpr uint32_t kAtomA = kRows * 128;  // 64 columns of 128 rows: 16 KB
constexpr uint32_t kAtomB = kH * 128;     // 64 columns of 256 rows: 32 KB
constexpr size_t kGemmSmem = 1024 + 4 * kAtomA + 4 * kAtomB + 64;

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const GemmTcParams P, const __grid_constant__ CUtensorMap mapA,
              const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapO,
              const __grid_constant__ CUtensorMap mapOT) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* base = tc_smem + ((1024u - (smem_u32(tc_smem) & 1023u)) & 1023u);
  unsigned char* As = base;               // 4 boxes of 16 KB
  unsigned char* Bs = base + 4 * kAtomA;  // 4 boxes of 32 KB
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + 4 * kAtomB);  // MMA completion
  uint64_t* tbar = bar + 1;                                       // TMA bytes landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & (kRows - 1), g = tid >> 7;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(tbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_warp = tmem + ((uint32_t)((warp & 3) * 32) << 16);

  const int64_t m_tiles = P.M / kRows;
  const int64_t items = m_tiles * P.splits;
  const int64_t ks = ((P.K + P.splits - 1) / P.splits + 63) / 64 * 64;  // K per split
  const bool b_resident = P.splits == 1 && P.K <= kH;
  auto row0_of = [&](int64_t mt_) { return mt_ * kRows; };
  auto range = [&](int64_t item, int64_t& kb, int64_t& ke) {
    kb = (item / m_tiles) * ks;
    ke = kb + ks < P.K ? kb + ks : P.K;
  };
  // one thread starts the TMA boxes of a chunk (kc a multiple of 64)
  auto issue = [&](int64_t item, int64_t c0, int kc, bool with_b) {
    if (tid != 0) return;
    const int boxes = kc / 64;
    bar_expect_tx(tbar, (uint32_t)boxes * (kAtomA + (with_b ? kAtomB : 0u)));
    const int y = (int)((item % m_tiles) * kRows);
    for (int a = 0; a < boxes; ++a) tma_load_2d(As + a * kAtomA, &mapA, (int)c0 + 64 * a, y, tbar);
    if (with_b)
      for (int a = 0; a < boxes; ++a) tma_load_2d(Bs + a * kAtomB, &mapB, (int)c0 + 64 * a, 0, tbar);
  };
  uint32_t parity = 0, tparity = 0;
  bool failed = false, b_loaded = false, prefetched = false;
  bool copy_failed = false, mma_failed = false;  // which bounded wait gave up

  for (int64_t item = blockIdx.x; item < items && !failed; item += gridDim.x) {
    int64_t kb, ke;
    range(item, kb, ke);
    if (kb >= ke) continue;  // an empty split (the same for every thread)
    const int64_t mt = item % m_tiles;
    float* const rowsum = P.rowsum;
    float row_acc = 0.f;
    for (int64_t c0 = kb; c0 < ke; c0 += kH) {
      const int kc = (int)(ke - c0 < kH ? ke - c0 : kH);
      if (!prefetched) issue(item, c0, kc, !(b_resident && b_loaded));
      prefetched = false;
      b_loaded = true;
      bool landed = bar_wait(tbar, tparity);  // the chunk's bytes are in shared memory
      if (!landed) landed = bar_wait(tbar, tparity);
      tparity ^= 1u;
      if (__syncthreads_or(!landed)) {
        if (tid == 0) atomicOr(P.err, 1u);
        failed = copy_failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (tid == 0) {
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll 1
        for (int k = 0; k < kc / 16; ++k) {
          // K step k: box k / 4, 32 (k % 4) bytes into each 128-byte row
          const uint32_t off_a = (uint32_t)(k >> 2) * kAtomA + 32u * (uint32_t)(k & 3);
          const uint32_t off_b = (uint32_t)(k >> 2) * kAtomB + 32u * (uint32_t)(k & 3);
          mma_bf16(tmem, sdesc_sw128(a0 + off_a), sdesc_sw128(b0 + off_b), kIdesc,
                   (c0 > kb || k > 0) ? 1u : 0u);
        }
        mma_commit(bar);
      }
      if (rowsum) {
        // while the MMAs run: thread (row r, half g) sums 4 of the 8 16-byte
        // chunks of its row in every box (the swizzle only permutes a row's
        // chunks, so the sum needs no unswizzling)
        for (int a = 0; a < kc / 64; ++a) {
          const unsigned char* rp = As + a * kAtomA + r * 128 + g * 64;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint4 q = *reinterpret_cast<const uint4*>(rp + 16 * c);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&w[e]);
              row_acc += __low2float(v) + __high2float(v);
            }
          }
        }
      }
      bool ok = bar_wait(bar, parity);
      if (!ok) ok = bar_wait(bar, parity);
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(P.err, 1u);
        failed = mma_failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (failed) break;
    // ---- epilogue, staged in the operand tiles (the MMAs are done with
    // them): row r of the tile, columns [128 g, 128 g + 128), written into
    // TMA store boxes in the 128-byte-swizzled layout (16-byte chunk j of a
    // 128-byte box row y at position j ^ (y % 8)) ----
    const int64_t row = mt * kRows + r;
    if (rowsum) atomicAdd(rowsum + row, row_acc);
    unsigned char* stage = base;
#pragma unroll 1
    for (int cc = 4 * g; cc < 4 * g + 4; ++cc) {
      uint32_t v[32];
      tmem_ld32(tmem_warp + (uint32_t)(cc * 32), v);
      const int col0 = cc * 32;
      if constexpr (EPI == GEMM_TC_ATOMIC) {
        // FP32 box cc (32 columns): row r, chunks q = 0..7
        unsigned char* rp = stage + cc * kAtomA + r * 128;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<uint4*>(rp + 16 * (q ^ (r & 7))) =
              make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        float f[32];
        if constexpr (EPI == GEMM_TC_BIAS_RELU) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 b4 = __ldg(reinterpret_cast<const float4*>(P.bias + col0 + j));
            f[j] = fmaxf(__uint_as_float(v[j]) + b4.x, 0.f);
            f[j + 1] = fmaxf(__uint_as_float(v[j + 1]) + b4.y, 0.f);
            f[j + 2] = fmaxf(__uint_as_float(v[j + 2]) + b4.z, 0.f);
            f[j + 3] = fmaxf(__uint_as_float(v[j + 3]) + b4.w, 0.f);
          }
        } else {
          const uint4* mrow = reinterpret_cast<const uint4*>(P.mask + row * P.ldm + col0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 mq = __ldg(mrow + q);
            const uint32_t mw[4] = {mq.x, mq.y, mq.z, mq.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
              const int j = 8 * q + 2 * e;
              f[j] = __low2float(m2) > 0.f ? __uint_as_float(v[j]) : 0.f;
              f[j + 1] = __high2float(m2) > 0.f ? __uint_as_float(v[j + 1]) : 0.f;
            }
          }
        }
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 32; j += 2) w[j / 2] = pack_bf16(f[j], f[j + 1]);
        // row-major box cc / 2 (64 columns): chunks 4 (cc % 2) .. + 3 of row r
        unsigned char* rp = stage + (cc >> 1) * kAtomA + r * 128;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * (cc & 1) + q;
          *reinterpret_cast<uint4*>(rp + 16 * (j ^ (r & 7))) =
              make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
        if (P.out_t) {
          // transposed boxes (64 tile rows x 256 columns): box r / 64, box row
          // = column c, element r % 64 of it
          const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(w);
          unsigned char* tb = stage + 4 * kAtomA + (r >> 6) * kAtomB;
          const int p = r & 63;
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int c = col0 + jj;
            *reinterpret_cast<__nv_bfloat16*>(tb + c * 128 + 16 * ((p >> 3) ^ (c & 7)) +
                                              2 * (p & 7)) = wb[jj];
          }
        }
      }
    }
    // the input layer's gradients need this tile's inputs: staged after the
    // output tiles (x rows of the tile, n_in <= 8 floats each)
    float* xs_tile = reinterpret_cast<float*>(stage + 4 * kAtomA + 2 * kAtomB);
    if (EPI == GEMM_TC_MASK && P.xin)
      for (int e = tid; e < kRows * P.n_in; e += kThreads) xs_tile[e] = P.xin[row0_of(mt) * P.n_in + e];
    // staging written (generic proxy) -> visible to the TMA (async proxy);
    // every TMEM read is done before the next item's MMAs overwrite it
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      const int y = (int)(mt * kRows);
      if constexpr (EPI == GEMM_TC_ATOMIC) {
        for (int b = 0; b < 8; ++b) tma_reduce_add_2d(&mapO, 32 * b, y, stage + b * kAtomA);
      } else {
        for (int b = 0; b < 4; ++b) tma_store_2d(&mapO, 64 * b, y, stage + b * kAtomA);
        if (P.out_t)
          for (int b = 0; b < 2; ++b)
            tma_store_2d(&mapOT, y + 64 * b, 0, stage + 4 * kAtomA + b * kAtomB);
      }
      bulk_commit();
    }
    if (EPI == GEMM_TC_MASK && P.xin) {
      // column tid of the staged bf16 tile against the tile's inputs, read
      // while the TMA stores it
      const int c = tid;
      const unsigned char* cb = stage + (c >> 6) * kAtomA + 2 * (c & 7);
      const int cj = (c & 63) >> 3;
      float aw[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, ab = 0.f;
      const int ni = P.n_in;
#pragma unroll 4
      for (int rr = 0; rr < kRows; ++rr) {
        const float z = __bfloat162float(
            *reinterpret_cast<const __nv_bfloat16*>(cb + rr * 128 + 16 * (cj ^ (rr & 7))));
        ab += z;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (i < ni) aw[i] = fmaf(z, xs_tile[rr * ni + i], aw[i]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < ni) atomicAdd(P.gw_in + c * ni + i, aw[i]);
      atomicAdd(P.gb_in + c, ab);
    }
    if (tid == 0) bulk_wait_read();  // the staging may be overwritten once the TMA has read it
    __syncthreads();
    // the staging overwrote the B tile: the next item copies B again, and its
    // first chunk is started now
    b_loaded = false;
    const int64_t next = item + gridDim.x;
    if (next < items) {
      int64_t nb, ne;
      range(next, nb, ne);
      if (nb < ne) {
        issue(next, nb, (int)(ne - nb < kH ? ne - nb : kH), true);
        prefetched = true;
        b_loaded = true;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (tid == 0) {
    // a timed-out wait: one more bounded wait for the copy or the MMAs still
    // in flight before the shared memory and TMEM are given up
    if (copy_failed) bar_wait(tbar, tparity ^ 1u);
    if (mma_failed) bar_wait(bar, parity ^ 1u);
    bulk_wait_all();  // every TMA store / reduction has completed
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}


// ---------------------------------------------------------------------------
// Weight gradients of the hidden layers: for up to kGemmBatch problems q,
// C_q[256][256] += A_q^T B_q with A_q = dz_l and B_q = h_{l-1} stored
// row-major [K][256] (K the batch), and rowsum_q[m] += sum_k A_q[k][m] (the
// bias gradient).  A work item is one problem's K range; the CTA computes the
// whole 256 x 256 output of it in 512 TMEM columns (two M = 128 halves against
// the same B chunk).  The K range streams through three shared-memory stages
// of 64 rows (A and B 64 x 256 bf16 each, 64 KB a stage) as TMA boxes of 64
// rows x 64 columns with the 128-byte swizzle, which the MMAs read as
// MN-major operands (the 256 columns contiguous, K the row).  The roles run
// independently, synchronised per stage by mbarriers only: one thread of
// warp 0 starts a stage's copies once its previous chunk's MMAs are done and
// its columns summed; one thread of warp 1 issues a chunk's 8 MMAs once it has
// landed and commits them to the stage's "MMAs done" barrier; warps 4..7 add
// the chunk's A columns to their column sums and arrive on its "summed"
// barrier.  After the item's last MMAs every warp takes part in the
// epilogue, which stages the FP32 output in the freed stages and adds it to C
// with TMA reduce-add, each CTA starting at a different box (the CTAs of a
// problem reduce into the same lines).
// ---------------------------------------------------------------------------
constexpr int kGemmBatch = 3;  // problems of one launch
constexpr int kWgStages = 3;
constexpr int kWgSumWarps = 4;  // column-sum warps: the last four
constexpr uint32_t kWgBox = 64 * 128;  // 64 rows x 64 bf16 columns: 8 KB
constexpr uint32_t kWgA = 4 * kWgBox;  // 64 rows x 256 columns: 32 KB
constexpr uint32_t kWgStage = 2 * kWgA;
constexpr size_t kWgSmem = 1024 + kWgStages * kWgStage + kWgSumWarps * kH * sizeof(float) +
                           (3 * kWgStages + 1) * 8 + 16;
constexpr uint32_t kWgTmemCols = 512;
// kind::f16 instruction descriptor as kIdesc with both operands MN-major
// (bits 15 and 16: A and B transposed)
constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);

// Descriptor of a 128-byte-swizzled MN-major operand made of the boxes above:
// 64 MN-contiguous elements per 128-byte row, one row per K; leading byte
// offset 8192 (the next box, 64 elements further along MN), stride byte
// offset 1024 (the next group of 8 K rows), version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(kWgBox >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Two bounded waits for the phase with the given parity.
__device__ __forceinline__ bool bar_wait2(uint64_t* bar, uint32_t parity) {
  return bar_wait(bar, parity) || bar_wait(bar, parity);
}

struct WgradMaps {
  CUtensorMap a[kGemmBatch], b[kGemmBatch], o[kGemmBatch];
  float* rowsum[kGemmBatch];
  int n_problems;
  int64_t K;       // columns of A and B (a multiple of 64)
  int64_t kchunk;  // K range of an item (a multiple of 64)
  int64_t splits;  // items per problem
  unsigned* err;
};

__global__ void __launch_bounds__(kThreads, 1) k_wgrad_tc(const __grid_constant__ WgradMaps W) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* base = tc_smem + ((1024u - (smem_u32(tc_smem) & 1023u)) & 1023u);
  float* colsum = reinterpret_cast<float*>(base + kWgStages * kWgStage);  // [kWgSumWarps][256]
  uint64_t* full = reinterpret_cast<uint64_t*>(colsum + kWgSumWarps * kH);  // bytes landed
  uint64_t* mdone = full + kWgStages;    // the stage's MMAs completed
  uint64_t* cdone = mdone + kWgStages;   // the stage's columns summed
  uint64_t* acc = cdone + kWgStages;     // every MMA of the item completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid & (kRows - 1), g = tid >> 7;
  constexpr int kSumWarp0 = kThreads / 32 - kWgSumWarps;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kWgTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kWgStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + s)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mdone + s)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(cdone + s)),
                   "r"(kWgSumWarps)
                   : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(acc)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_warp = tmem + ((uint32_t)((warp & 3) * 32) << 16);

  const int64_t items = W.splits * W.n_problems;
  // chunks started in the CTA's earlier items (stage of chunk gc: gc % 3, its
  // use of that stage: gc / 3) and items finished (phase of acc)
  uint32_t gbase = 0, nitem = 0;
  // for the drain after a timed-out wait: chunks copied (producer thread),
  // chunks committed and whether an acc commit is unwaited (MMA thread)
  uint32_t n_issued = 0, n_committed = 0;
  bool acc_pending = false, failed = false;
  for (int64_t item = blockIdx.x; item < items && !failed; item += gridDim.x) {
    const int q = (int)(item / W.splits);
    const int64_t kb = (item % W.splits) * W.kchunk;
    const int64_t ke = kb + W.kchunk < W.K ? kb + W.kchunk : W.K;
    if (kb >= ke) continue;  // the same for every thread
    const int nch = (int)((ke - kb) / 64);
    bool ok = true;
    // columns 8 lane .. + 7 of A summed over the item's rows k with
    // k % 4 = (column-sum warp index)
    float racc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) racc[e] = 0.f;
    if (warp == 0) {
      if (lane == 0) {
        // producer: a stage is refilled once its previous chunk's MMAs are
        // done and its columns summed
        for (int c = 0; c < nch; ++c) {
          const uint32_t gc = gbase + (uint32_t)c, s = gc % kWgStages, u = gc / kWgStages;
          if (u > 0 && !(bar_wait2(mdone + s, (u - 1) & 1u) && bar_wait2(cdone + s, (u - 1) & 1u))) {
            ok = false;
            break;
          }
          unsigned char* st = base + s * kWgStage;
          bar_expect_tx(full + s, kWgStage);
          const int y = (int)(kb + 64 * c);
          for (int j = 0; j < 4; ++j) tma_load_2d(st + j * kWgBox, &W.a[q], 64 * j, y, full + s);
          for (int j = 0; j < 4; ++j)
            tma_load_2d(st + kWgA + j * kWgBox, &W.b[q], 64 * j, y, full + s);
          n_issued = gc + 1;
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        // MMA issuer: a chunk's 8 MMAs as soon as it has landed
        for (int c = 0; c < nch; ++c) {
          const uint32_t gc = gbase + (uint32_t)c, s = gc % kWgStages, u = gc / kWgStages;
          if (!bar_wait2(full + s, u & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t a0 = smem_u32(base + s * kWgStage), b0 = a0 + kWgA;
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_bf16(tmem + 256u * h, sdesc_mn_sw128(a0 + 2u * kWgBox * h + 2048u * k),
                       sdesc_mn_sw128(b0 + 2048u * k), kIdescMN, (c > 0 || k > 0) ? 1u : 0u);
          mma_commit(mdone + s);
          n_committed = gc + 1;
        }
        if (ok) {
          mma_commit(acc);  // arrives once every MMA issued so far has completed
          acc_pending = true;
        }
      }
    } else if (warp >= kSumWarp0) {
      // column sums: lane l adds columns 8 l .. 8 l + 7 (box l / 8, 16-byte
      // chunk l % 8 XOR-ed with the row's k % 8 by the swizzle) of the rows
      // k = sw + 4 j; a warp's load covers one row's 512 bytes
      const int sw = warp - kSumWarp0;
      for (int c = 0; c < nch; ++c) {
        const uint32_t gc = gbase + (uint32_t)c, s = gc % kWgStages, u = gc / kWgStages;
        if (!__all_sync(0xffffffffu, bar_wait2(full + s, u & 1u))) {
          ok = false;
          break;
        }
        const unsigned char* cp = base + s * kWgStage + (lane >> 3) * kWgBox;
#pragma unroll
        for (int j = 0; j < 64 / kWgSumWarps; ++j) {
          const int k = sw + kWgSumWarps * j;
          const uint4 v = *reinterpret_cast<const uint4*>(cp + k * 128 + (((lane & 7) ^ (k & 7)) << 4));
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 p = *reinterpret_cast<const __nv_bfloat162*>(&w[e]);
            racc[2 * e] += __low2float(p);
            racc[2 * e + 1] += __high2float(p);
          }
        }
        __syncwarp();
        if (lane == 0) bar_arrive(cdone + s);
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // every MMA of the item has completed: the accumulators are final
    const bool aok = bar_wait2(acc, nitem & 1u);
    if (warp == 1 && lane == 0 && aok) acc_pending = false;
    if (warp >= kSumWarp0) {
      float4* cs = reinterpret_cast<float4*>(colsum + (warp - kSumWarp0) * kH + 8 * lane);
      cs[0] = make_float4(racc[0], racc[1], racc[2], racc[3]);
      cs[1] = make_float4(racc[4], racc[5], racc[6], racc[7]);
    }
    if (__syncthreads_or(!aok)) {
      failed = true;
      break;
    }
    ++nitem;
    gbase += (uint32_t)nch;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (W.rowsum[q]) {
      // column tid: the row classes' sums in a fixed order
      float cs = 0.f;
#pragma unroll
      for (int k = 0; k < kWgSumWarps; ++k) cs += colsum[k * kH + tid];
      atomicAdd(W.rowsum[q] + tid, cs);
    }
    // ---- epilogue: each half as eight FP32 boxes of 32 columns x 128 rows
    // (128-byte swizzle) in the freed stages, added to C by TMA; the CTA's
    // first half and first box rotate with its index ----
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
      const int h = hh ^ (int)((blockIdx.x >> 3) & 1u);
#pragma unroll 1
      for (int cc = 4 * g; cc < 4 * g + 4; ++cc) {
        uint32_t v[32];
        tmem_ld32(tmem_warp + 256u * h + (uint32_t)(cc * 32), v);
        unsigned char* rp = base + cc * kAtomA + r * 128;
#pragma unroll
        for (int qq = 0; qq < 8; ++qq)
          *reinterpret_cast<uint4*>(rp + 16 * (qq ^ (r & 7))) =
              make_uint4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (tid == 0) {
        for (int b0 = 0; b0 < 8; ++b0) {
          const int b = (b0 + (int)blockIdx.x) & 7;
          tma_reduce_add_2d(&W.o[q], 32 * b, 128 * h, base + b * kAtomA);
        }
        bulk_commit();
        bulk_wait_read();  // the staging may be overwritten once the TMA has read it
      }
      __syncthreads();
    }
  }
  if (failed) {
    if (tid == 0) atomicOr(W.err, 1u);
    // before the shared memory and TMEM are given up: one more bounded wait
    // for the copies (producer) and MMAs (issuer) possibly still in flight
    if (warp == 0 && lane == 0)
      for (uint32_t gc = n_issued > kWgStages ? n_issued - kWgStages : 0; gc < n_issued; ++gc)
        bar_wait(full + gc % kWgStages, (gc / kWgStages) & 1u);
    if (warp == 1 && lane == 0) {
      for (uint32_t gc = n_committed > kWgStages ? n_committed - kWgStages : 0; gc < n_committed;
           ++gc)
        bar_wait(mdone + gc % kWgStages, (gc / kWgStages) & 1u);
      if (acc_pending) bar_wait(acc, nitem & 1u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (tid == 0) bulk_wait_all();  // every TMA reduction has completed
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kWgTmemCols)
                 : "memory");
}

}  // namespace

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor map of a row-major matrix (rows x cols, leading dimension ld
// elements; bf16 or FP32) in boxes of 128 bytes of a row (64 bf16 or 32 FP32)
// x box_rows rows, 128-byte swizzle.  Maps are cached by (address, type,
// shape, box): the training step reuses a few fixed buffers.
bool tensor_map(const void* base, bool f32, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                CUtensorMap* out) {
  struct Entry {
    const void* base;
    bool f32;
    int64_t rows, cols, ld;
    int box_rows;
    CUtensorMap map;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.base == base && e.f32 == f32 && e.rows == rows && e.cols == cols && e.ld == ld &&
        e.box_rows == box_rows) {
      *out = e.map;
      return true;
    }
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  Entry e{base, f32, rows, cols, ld, box_rows, {}};
  const size_t esz = f32 ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  if (fn(&e.map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  if (cache.size() >= 64) cache.erase(cache.begin());
  cache.push_back(e);
  *out = e.map;
  return true;
}

}  // namespace

cudaError_t gemm_tc(int epi, const GemmTcParams& p, int device, int sm_count, cudaStream_t s) {
  // TMA: 16-byte aligned bases, row pitches a multiple of 16 bytes; boxes of
  // 64 columns, so K is a multiple of 64 (every box starts on a 128-byte
  // boundary of its row)
  const bool aligned = ((uintptr_t)p.A % 16 == 0) && ((uintptr_t)p.B % 16 == 0) &&
                       p.lda % 8 == 0 && p.ldb % 8 == 0 && p.lda >= p.K && p.ldb >= p.K;
  bool ok = aligned && p.M > 0 && p.M % kRows == 0 && p.K > 0 && p.K % 64 == 0 && p.splits >= 1 &&
            p.err;
  if (epi == GEMM_TC_ATOMIC)
    ok = ok && p.out_f && (uintptr_t)p.out_f % 16 == 0 && p.ldf % 4 == 0 && p.ldf >= kH;
  else
    ok = ok && p.out && (uintptr_t)p.out % 16 == 0 && p.ldo % 8 == 0 && p.ldo >= kH &&
         (!p.out_t || ((uintptr_t)p.out_t % 16 == 0 && p.ldot % 8 == 0 && p.ldot >= p.M)) &&
         (epi == GEMM_TC_BIAS_RELU ? (p.bias && (uintptr_t)p.bias % 16 == 0)
                                   : (p.mask && (uintptr_t)p.mask % 16 == 0 && p.ldm % 8 == 0));
  if (p.xin) ok = ok && epi == GEMM_TC_MASK && p.n_in >= 1 && p.n_in <= 8 && p.gw_in && p.gb_in;
  if (!ok || epi < GEMM_TC_BIAS_RELU || epi > GEMM_TC_ATOMIC) return cudaErrorInvalidValue;
  // operand maps (loads) and output maps (stores / reductions of the tile)
  CUtensorMap mapA, mapB, mapO, mapOT;
  memset(&mapOT, 0, sizeof(mapOT));
  bool maps = tensor_map(p.A, false, p.M, p.K, p.lda, kRows, &mapA) &&
              tensor_map(p.B, false, kH, p.K, p.ldb, kH, &mapB);
  if (epi == GEMM_TC_ATOMIC) {
    maps = maps && tensor_map(p.out_f, true, p.M, kH, p.ldf, kRows, &mapO);
  } else {
    maps = maps && tensor_map(p.out, false, p.M, kH, p.ldo, kRows, &mapO);
    if (p.out_t) maps = maps && tensor_map(p.out_t, false, kH, p.M, p.ldot, kH, &mapOT);
  }
  if (!maps) return cudaErrorInvalidValue;
  auto k = epi == GEMM_TC_BIAS_RELU ? k_gemm_tc<GEMM_TC_BIAS_RELU>
           : epi == GEMM_TC_MASK    ? k_gemm_tc<GEMM_TC_MASK>
                                    : k_gemm_tc<GEMM_TC_ATOMIC>;
  // the shared-memory opt-in is a per-device attribute of each kernel: set once
  static std::atomic<uint64_t> set_mask[3];
  const uint64_t bit = device >= 0 && device < 64 ? (1ull << device) : 0ull;
  if (!bit || !(set_mask[epi].load() & bit)) {
    cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    if (e != cudaSuccess) return e;
    set_mask[epi].fetch_or(bit);
  }
  const int64_t items = p.M / kRows * p.splits;
  const int64_t grid = items < sm_count ? items : sm_count;
  k<<<(unsigned)grid, kThreads, kGemmSmem, s>>>(p, mapA, mapB, mapO, mapOT);
  return cudaGetLastError();
}

cudaError_t wgrad_tc(const GemmTcParams* ps, int np, int sm_count, cudaStream_t s) {
  if (np < 1 || np > kGemmBatch) return cudaErrorInvalidValue;
  WgradMaps W;
  memset(&W, 0, sizeof(W));
  W.n_problems = np;
  W.K = ps[0].K;
  W.err = ps[0].err;
  for (int q = 0; q < np; ++q) {
    const GemmTcParams& p = ps[q];
    // A and B row-major [K][256]: 16-byte aligned bases and row pitches
    const bool ok = p.M == kH && p.K == W.K && p.K > 0 && p.K % 64 == 0 && p.err == W.err &&
                    p.err && ((uintptr_t)p.A % 16 == 0) && ((uintptr_t)p.B % 16 == 0) &&
                    p.lda % 8 == 0 && p.ldb % 8 == 0 && p.lda >= kH && p.ldb >= kH && p.out_f &&
                    (uintptr_t)p.out_f % 16 == 0 && p.ldf % 4 == 0 && p.ldf >= kH;
    if (!ok) return cudaErrorInvalidValue;
    W.rowsum[q] = p.rowsum;
    if (!tensor_map(p.A, false, p.K, kH, p.lda, 64, &W.a[q]) ||
        !tensor_map(p.B, false, p.K, kH, p.ldb, 64, &W.b[q]) ||
        !tensor_map(p.out_f, true, kH, kH, p.ldf, kRows, &W.o[q]))
      return cudaErrorInvalidValue;
  }
  // one wave: at most sm_count items, K ranges a multiple of 64
  const int64_t per = sm_count / np > 1 ? sm_count / np : 1;
  W.kchunk = ((W.K + per - 1) / per + 63) / 64 * 64;
  W.splits = (W.K + W.kchunk - 1) / W.kchunk;
  static std::atomic<uint64_t> set_mask{0};
  int device = 0;
  cudaGetDevice(&device);
  const uint64_t bit = device >= 0 && device < 64 ? (1ull << device) : 0ull;
  if (!bit || !(set_mask.load() & bit)) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    if (e != cudaSuccess) return e;
    set_mask.fetch_or(bit);
  }
  const int64_t items = W.splits * np;
  const int64_t grid = items < sm_count ? items : sm_count;
  k_wgrad_tc<<<(unsigned)grid, kThreads, kWgSmem, s>>>(W);
  return cudaGetLastError();
}

size_t mlp_tc_weight_image_elems() { return (size_t)kH * kH; }

bool mlp_tc_supported(int n_in, int hidden, int n_hidden, int n_out) {
  return hidden == kH && n_in >= 1 && n_in <= 8 && n_out == 3 && n_hidden >= 2 &&
         n_hidden - 1 <= kMlpTcMaxGemm;
}

template <bool TRAIN>
cudaError_t launch_forward_tc(const MlpTcParams& p, int sm_count, cudaStream_t s) {
  // weight images: one bulk copy each (16-byte aligned)
  if (p.n_gemm < 1 || p.n_gemm > kMlpTcMaxGemm) return cudaErrorInvalidValue;
  for (int l = 0; l < p.n_gemm; ++l)
    if (!p.Wimg[l] || (uintptr_t)p.Wimg[l] % 16 != 0) return cudaErrorInvalidValue;
  auto k = p.n_in == 4 ? k_mlp_forward_tc<4, TRAIN> : k_mlp_forward_tc<0, TRAIN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  int64_t grid = p.n_tiles < sm_count ? p.n_tiles : sm_count;
  if (grid < 1) return cudaSuccess;
  k<<<(unsigned)grid, kThreads, kSmem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t mlp_forward_tc(const MlpTcParams& p, int sm_count, cudaStream_t s) {
  return launch_forward_tc<false>(p, sm_count, s);
}

cudaError_t mlp_forward_tc_train(const MlpTcParams& p, int sm_count, cudaStream_t s) {
  return launch_forward_tc<true>(p, sm_count, s);
}

const void* mlp_train_tc_kernel(int n_in) {
  return n_in == 4 ? reinterpret_cast<const void*>(k_mlp_train_tc<4>)
                   : reinterpret_cast<const void*>(k_mlp_train_tc<0>);
}

cudaError_t mlp_train_tc(const MlpTrainTcParams& p, int sm_count, cudaStream_t s) {
  auto k = p.n_in == 4 ? k_mlp_train_tc<4> : k_mlp_train_tc<0>;
  cudaError_t e =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
  if (e != cudaSuccess) return e;
  int64_t grid = p.n_tiles < sm_count ? p.n_tiles : sm_count;
  if (grid < 1) return cudaSuccess;
  // weight images: one bulk copy each (16-byte aligned)
  for (int l = 0; l < kMlpTrainGemm; ++l)
    if (!p.Wimg[l] || !p.WimgT[l] || (uintptr_t)p.Wimg[l] % 16 != 0 ||
        (uintptr_t)p.WimgT[l] % 16 != 0)
      return cudaErrorInvalidValue;
  // the inputs of GEMMs 0 .. 5: h_0, h_1, h_2, dz_3, dz_2, dz_1 (row-major
  // [n][256], 16-byte aligned: TMA stores of 64-column boxes)
  const __nv_bfloat16* outs[2 * kMlpTrainGemm] = {p.h[0], p.h[1], p.h[2], p.dz[3], p.dz[2], p.dz[1]};
  TrainStoreMaps T;
  memset(&T, 0, sizeof(T));
  for (int i = 0; i < 2 * kMlpTrainGemm; ++i)
    if (!outs[i] || (uintptr_t)outs[i] % 16 != 0 ||
        !tensor_map(outs[i], false, p.n, kH, kH, kRows, &T.out[i]))
      return cudaErrorInvalidValue;
  k<<<(unsigned)grid, kThreads, kTrainSmem, s>>>(p, T);
  return cudaGetLastError();
}

}  // namespace crp
