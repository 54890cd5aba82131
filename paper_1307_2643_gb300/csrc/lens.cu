// lens.cu -- galactic lens: build by back-tracking, apply, arrival maps.
//
// CRPropa 3.0 (Sect. 4, "Galactic propagation") maps the directions of
// cosmic rays at the border of the Galaxy to the directions observed at
// Earth with a set of transformation matrices, one per energy bin, built by
// tracking through a galactic field model.  Here, per rigidity bin b and
// HEALPix RING border pixel j, the lens keeps the multiset of Earth pixels i
// of the back-tracked samples that left the Galaxy through j (a column of
// the count matrix N_b[i, j]), sorted ascending, plus the largest column
// count of each bin.  Apply: observed with probability count_j / max_b
// (M_b = N_b / max_j sum_i N_b[i, j]; the rest is shadowed), then a
// uniformly chosen sample of the column gives the Earth pixel.
#include <math.h>
#include <string.h>

#include <cmath>

#include <new>
#include <vector>

#include "crp_internal.cuh"
#include "device_common.cuh"

namespace crp {
void context_view(const crp_context* c, const int32_t** status, const double** E, uint64_t* n,
                  int* device);
void context_pool(const crp_context* c, DevState* st, uint64_t* n, int* device, uint64_t* seed);
void context_scratch(const crp_context* c, uint32_t** list, unsigned long long** counter);
}  // namespace crp

using namespace crp;

struct crp_lens {
  int device;
  int32_t nside, n_bins;
  double r_lo, r_hi;
  int64_t npix, n_cols, n_entries;
  uint32_t* col_start;  // n_cols + 1
  uint32_t* entries;    // n_entries Earth pixels
  uint32_t* max_count;  // n_bins
};

namespace {

constexpr uint32_t kNotApplied = 0xFFFFFFFFu;
constexpr uint32_t kNotObserved = 0xFFFFFFFEu;
constexpr uint32_t kNoKey = 0xFFFFFFFFu;
constexpr int kScanBlock = 1024;

int blocks(uint64_t n, int b) {
  const uint64_t g = (n + b - 1) / b;
  return (int)(g < 1 ? 1 : (g > 65536 ? 65536 : g));
}

// Per back-tracked sample: column key b * npix + j (border pixel of the
// antiparticle's direction) for samples that reached the border, and the
// Earth pixel i of its launch direction.
__global__ void k_lens_keys(DevState st, uint64_t n, const int32_t* bin, int64_t nside,
                            int64_t npix, uint32_t* key, uint32_t* earth, uint32_t* counts) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    earth[k] = (uint32_t)healpix_ring_pixel_guarded<false>(nside, st.ux0[k], st.uy0[k], st.uz0[k]);
    if (st.status[k] != CRP_AT_BORDER) {
      key[k] = kNoKey;
      continue;
    }
    const int64_t j = healpix_ring_pixel_guarded<false>(nside, st.ux[k], st.uy[k], st.uz[k]);
    const uint32_t c = (uint32_t)((int64_t)bin[k] * npix + j);
    key[k] = c;
    atomicAdd(counts + c, 1u);
  }
}

// Exclusive scan of n uint32 in place: block scans, scan of block sums,
// add-back.  out[n] receives the total.
__global__ void k_scan_blocks(uint32_t* v, uint64_t n, uint32_t* block_sums) {
  __shared__ uint32_t sh[kScanBlock];
  const uint64_t i = blockIdx.x * (uint64_t)kScanBlock + threadIdx.x;
  const uint32_t x = i < n ? v[i] : 0u;
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const uint32_t t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0u;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) v[i] = sh[threadIdx.x] - x;  // exclusive
  if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_sums(uint32_t* sums, int nb, uint32_t* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t run = 0;
  for (int b = 0; b < nb; ++b) {
    const uint32_t v = sums[b];
    sums[b] = run;
    run += v;
  }
  *total = run;
}

__global__ void k_scan_add(uint32_t* v, uint64_t n, const uint32_t* sums) {
  const uint64_t i = blockIdx.x * (uint64_t)kScanBlock + threadIdx.x;
  if (i < n) v[i] += sums[blockIdx.x];
}

__global__ void k_lens_scatter(const uint32_t* key, const uint32_t* earth, uint64_t n,
                               uint32_t* fill, uint32_t* entries) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (key[k] == kNoKey) continue;
    entries[atomicAdd(fill + key[k], 1u)] = earth[k];
  }
}

// Canonical order inside each column (ascending Earth pixel), so the lens
// does not depend on the order the samples were scattered in.
__global__ void k_lens_sort_columns(const uint32_t* col_start, int64_t n_cols, uint32_t* entries) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cols;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t a = col_start[c], b = col_start[c + 1];
    for (uint32_t i = a + 1; i < b; ++i) {
      const uint32_t v = entries[i];
      uint32_t j = i;
      while (j > a && entries[j - 1] > v) {
        entries[j] = entries[j - 1];
        --j;
      }
      entries[j] = v;
    }
  }
}

__global__ void k_lens_max(const uint32_t* col_start, int64_t npix, int n_bins, uint32_t* mx) {
  __shared__ uint32_t sh[256];
  const int b = blockIdx.x;
  if (b >= n_bins) return;
  uint32_t m = 0;
  for (int64_t j = threadIdx.x; j < npix; j += blockDim.x) {
    const int64_t c = (int64_t)b * npix + j;
    const uint32_t cnt = col_start[c + 1] - col_start[c];
    m = cnt > m ? cnt : m;
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < (unsigned)s) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) mx[b] = sh[0];
}

__device__ __forceinline__ bool pick(int what, int status) {
  switch (what) {
    case CRP_COLLECT_ALL: return true;
    case CRP_COLLECT_FINISHED: return status != CRP_ACTIVE;
    case CRP_COLLECT_DETECTED: return status == CRP_DETECTED;
    case CRP_COLLECT_ACTIVE: return status == CRP_ACTIVE;
    case CRP_COLLECT_AT_BORDER: return status == CRP_AT_BORDER;
  }
  return false;
}

// Rigidity bin of R = E / Z in binary64: floor((ln R - ln r_lo) * inv_dlg),
// clamped to [0, n_bins - 1].
__device__ __forceinline__ int64_t lens_bin_f64(double E, int Z, double lg_lo, double inv_dlg,
                                                int n_bins) {
  const double R = E / (double)Z;
  const double t = (series_log(R) - lg_lo) * inv_dlg;
  double bf = floor(t);
  if (!(bf >= 0.0)) bf = 0.0;
  if (bf > (double)(n_bins - 1)) bf = (double)(n_bins - 1);
  return (int64_t)bf;
}

// The same bin from t = log2(R / r_lo) * inv_dlg ln 2 in binary32, when its
// error bound leaves no doubt.  Error of t against the exact value: R / r_lo
// formed in binary32 from E truncated to binary32 (2^-23), 1 / r_lo and the
// product (2^-24 each) and __fdividef (2 ulp), 4.8e-7 relative in all, so
// inv_dlg * 4.8e-7 on t; __log2f (CUDA's bound: 2^-22 absolute on [0.5, 2],
// 2 ulp elsewhere): inv_dlg * 1.7e-7 + |t| * 2.4e-7; the factor inv_dlg ln 2
// and the product (2^-24 each): |t| * 1.2e-7.  Below inv_dlg * 6.5e-7 + |t| *
// 3.6e-7 in all; the guard inv_dlg * 1e-5 + |t| * 1.5e-6 + 1e-6 is 15x and
// 4x that.  False when undecided.
__device__ __forceinline__ bool lens_bin_f32(double E, int Z, float inv_rlo_f, float inv_f,
                                             float inv2_f, int n_bins, int* b) {
  const float x = __fdividef(f32_trunc(E) * inv_rlo_f, (float)Z);
  const float t = __log2f(x) * inv2_f;
  const float g = inv_f * 1e-5f + fabsf(t) * 1.5e-6f + 1e-6f;
  if (t + g < 0.f) {
    *b = 0;
    return true;
  }
  if (t - g >= (float)(n_bins - 1)) {
    *b = n_bins - 1;
    return true;
  }
  return floor_sure(t, g, b);
}

// Apply the lens (Sect. 4, transformation matrices by rigidity bin): bin b
// of R = E / Z, column j = pixel of the arrival direction -u; with the two
// uniforms (u1, u2) of Philox draw 0, tag 3 of the candidate's id it is
// observed when u1 * max_count_b < count_j, at the Earth pixel
// entries[min(floor(u2 * count_j), count_j - 1)] of the column.  Each integer
// decision is first taken in binary32 with a guard from its error bound and
// in binary64 only inside the guard, so the result is the binary64 one.
// Lens application in two passes.  The first decides, in binary32, every
// candidate whose decisions (rigidity bin, border pixel, observed or not,
// pick) are all outside their guard bands -- each such decision equals the
// binary64 one -- and appends the others to a list (one atomic per warp).
// The second runs the binary64 decisions over that list with full warps, so
// no warp of the first pass waits on binary64 code.
struct LensArgs {
  uint64_t seed;
  int64_t nside, npix;
  int n_bins, use_f32;
  double lg_lo, inv_dlg;
  float inv_rlo_f, inv_f, inv2_f;  // 1 / r_lo, inv_dlg and inv_dlg ln 2 in binary32
  const uint32_t* col_start;
  const uint32_t* entries;
  const uint32_t* max_count;
};

// The Earth pixel from a column (start, count): observed when u1 max_count <
// count, then entry floor(u2 count) (binary64 decisions).
__device__ __forceinline__ uint32_t lens_pick_f64(const LensArgs& a, const Philox4& w,
                                                  uint32_t start, uint32_t count, uint32_t mxi) {
  if (!(u01_open(w.v0, w.v1) * (double)mxi < (double)count)) return kNotObserved;
  int64_t pk = (int64_t)(u01_open(w.v2, w.v3) * (double)count);
  if (pk > (int64_t)count - 1) pk = (int64_t)count - 1;
  return a.entries[start + pk];
}

// The pick in binary32 when its guards leave no doubt (the binary64 pick's
// result then); false when undecided.  u1 lies in [h1, h1 + 2^-24) with h1
// its top 24 bits (exact in binary32): u1 * max_count is known to 2.4e-7 *
// max_count, and likewise u2 * count.
__device__ __forceinline__ bool lens_pick_try_f32(const LensArgs& a, const Philox4& w,
                                                  uint32_t start, uint32_t count, uint32_t mxi,
                                                  uint32_t* out) {
  const float mxf = (float)mxi, cf = (float)count;
  const float p1 = (float)(w.v1 >> 8) * 5.9604644775390625e-8f * mxf;
  if (!(fabsf(p1 - cf) > 2e-6f * mxf)) return false;
  if (!(p1 < cf)) {
    *out = kNotObserved;
    return true;
  }
  const float p2 = (float)(w.v3 >> 8) * 5.9604644775390625e-8f * cf;
  int pk32;
  if (!floor_sure(p2, 2e-6f * cf, &pk32)) return false;
  *out = a.entries[start + pk32];
  return true;
}

// The binary32 decisions of one selected candidate: its lens pixel written
// when every decision is sure; false (written nothing) when it must go to
// the binary64 pass.  The candidate's uniforms do not depend on the lens, so
// Philox runs before the column lookups, while they are in flight.
__device__ __forceinline__ bool lens_decide_f32(const LensArgs& a, int Z, double E, double ux,
                                                double uy, double uz, uint64_t id,
                                                uint32_t* pixel_out) {
  if (Z <= 0) {
    *pixel_out = kNotApplied;
    return true;
  }
  int b;
  int64_t j;
  bool sure = a.use_f32 && lens_bin_f32(E, Z, a.inv_rlo_f, a.inv_f, a.inv2_f, a.n_bins, &b);
  sure = sure && healpix_ring_pixel_try<true>(a.nside, ux, uy, uz, &j);
  if (!sure) return false;
  // column keys are 32-bit (the lens build checks n_bins * npix < 2^32)
  const uint32_t col = (uint32_t)b * (uint32_t)a.npix + (uint32_t)j;
  const uint32_t start = a.col_start[col];
  const uint32_t count = a.col_start[col + 1] - start;
  const uint32_t mxi = a.max_count[b];
  const Philox4 w = draw4(a.seed, 3u, id, 0u);
  uint32_t out = kNotObserved;
  if (count > 0 && !lens_pick_try_f32(a, w, start, count, mxi, &out)) return false;
  *pixel_out = out;
  return true;
}

// First pass, a persistent grid: each thread walks its candidates with a
// stride of the grid, holding the next candidate's inputs in registers while
// it decides the current one (its status two candidates ahead, so that the
// other inputs are read only for selected candidates without waiting), and
// appends the undecided ones to the list (one atomic per warp).  WHAT is the
// status filter (for CRP_COLLECT_ALL no status is read); indices are 32-bit
// (the host checks n < 2^31, as the list of undecided indices needs).
template <int WHAT>
__global__ void k_lens_apply_f32(DevState st, uint32_t n, LensArgs a, uint32_t* fallback,
                                 unsigned long long* n_fallback) {
  constexpr int what = WHAT;
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t base = blockIdx.x * blockDim.x;
  uint32_t k = base + threadIdx.x;
  // current candidate
  // the candidate arrays are read once: streaming loads (evict first), so
  // that the lens tables stay in L2
  bool sel = k < n && pick(what, __ldcs(st.status + k));
  int Z = 0;
  double E = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
  uint64_t id = 0;
  if (sel) {
    Z = __ldcs(st.Z + k);
    E = __ldcs(st.E + k);
    ux = __ldcs(st.ux + k);
    uy = __ldcs(st.uy + k);
    uz = __ldcs(st.uz + k);
    id = __ldcs(reinterpret_cast<const unsigned long long*>(st.id) + k);
  }
  // the next candidate's status
  bool sel_next = k + stride < n && pick(what, __ldcs(st.status + k + stride));
  for (; base < n; base += stride) {
    const uint32_t kn = k + stride, knn = kn + stride;
    int Z2 = 0;
    double E2 = 0.0, ux2 = 0.0, uy2 = 0.0, uz2 = 0.0;
    uint64_t id2 = 0;
    if (sel_next) {
      Z2 = __ldcs(st.Z + kn);
      E2 = __ldcs(st.E + kn);
      ux2 = __ldcs(st.ux + kn);
      uy2 = __ldcs(st.uy + kn);
      uz2 = __ldcs(st.uz + kn);
      id2 = __ldcs(reinterpret_cast<const unsigned long long*>(st.id) + kn);
    }
    const bool sel_nn = knn < n && pick(what, __ldcs(st.status + knn));
    bool defer = false;
    if (sel) {
      uint32_t out;
      defer = !lens_decide_f32(a, Z, E, ux, uy, uz, id, &out);
      if (!defer) __stcs(st.lens_pixel + k, out);
    }
    // append the undecided candidates of this warp to the list
    const unsigned m = __ballot_sync(0xffffffffu, defer);
    if (m) {
      unsigned long long slot = 0;
      const int leader = __ffs(m) - 1;
      if (lane == leader) slot = atomicAdd(n_fallback, (unsigned long long)__popc(m));
      slot = __shfl_sync(0xffffffffu, slot, leader);
      if (defer) fallback[slot + __popc(m & ((1u << lane) - 1u))] = k;
    }
    k = kn;
    sel = sel_next;
    sel_next = sel_nn;
    Z = Z2;
    E = E2;
    ux = ux2;
    uy = uy2;
    uz = uz2;
    id = id2;
  }
}

__global__ void k_lens_apply_f64(DevState st, LensArgs a, const uint32_t* fallback,
                                 const unsigned long long* n_fallback) {
  const uint64_t m = *n_fallback;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = fallback[i];
    // each decision again in binary32 first (deterministic: the same sure
    // results as the first pass); binary64 only for those inside their guard
    const double E = st.E[k], ux = st.ux[k], uy = st.uy[k], uz = st.uz[k];
    const int Z = st.Z[k];
    int b32;
    const int64_t b = a.use_f32 && lens_bin_f32(E, Z, a.inv_rlo_f, a.inv_f, a.inv2_f, a.n_bins, &b32)
                          ? (int64_t)b32
                          : lens_bin_f64(E, Z, a.lg_lo, a.inv_dlg, a.n_bins);
    int64_t j;
    if (!healpix_ring_pixel_try<true>(a.nside, ux, uy, uz, &j))
      j = healpix_ring_pixel(a.nside, -ux, -uy, -uz);
    const int64_t col = b * a.npix + j;
    const uint32_t start = a.col_start[col];
    const uint32_t count = a.col_start[col + 1] - start;
    uint32_t out = kNotObserved;
    if (count > 0) {
      const Philox4 w = draw4(a.seed, 3u, st.id[k], 0u);
      const uint32_t mxi = a.max_count[b];
      if (!lens_pick_try_f32(a, w, start, count, mxi, &out))
        out = lens_pick_f64(a, w, start, count, mxi);
    }
    st.lens_pixel[k] = out;
  }
}

__global__ void k_hist_healpix(DevState st, uint64_t n, int what, int64_t nside, int source,
                               unsigned long long* bins) {
  const uint64_t npix = 12ull * nside * nside;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (!pick(what, st.status[k])) continue;
    uint64_t p;
    if (source == 0)
      p = (uint64_t)healpix_ring_pixel_guarded<true>(nside, st.ux[k], st.uy[k], st.uz[k]);
    else
      p = st.lens_pixel[k];
    if (p < npix) atomicAdd(bins + p, 1ull);
  }
}

crp_status scan_inplace(uint32_t* v, uint64_t n, uint32_t* total, cudaStream_t s) {
  const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
  uint32_t* sums = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * (nb + 1)));
  if (!sums) {
    set_error("lens: scan workspace allocation failed");
    return CRP_E_OOM;
  }
  k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, s>>>(v, n, sums);
  k_scan_sums<<<1, 1, 0, s>>>(sums, (int)nb, total);
  k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(v, n, sums);
  const cudaError_t e = cudaStreamSynchronize(s);
  dev_free(sums);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "lens: scan");
}

void lens_free(crp_lens* L) {
  if (!L) return;
  dev_free(L->col_start);
  dev_free(L->entries);
  dev_free(L->max_count);
  delete L;
}


// A lens shell with zeroed column counts (col_start doubles as the count
// array until lens_columns scans it).
crp_lens* lens_alloc(int device, const crp_lens_desc* d, int64_t npix, int64_t n_cols) {
  crp_lens* L = new (std::nothrow) crp_lens;
  if (!L) return nullptr;
  memset(L, 0, sizeof(*L));
  L->device = device;
  L->nside = d->nside;
  L->n_bins = d->n_bins;
  L->r_lo = d->r_lo;
  L->r_hi = d->r_hi;
  L->npix = npix;
  L->n_cols = n_cols;
  L->col_start = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * (n_cols + 1)));
  L->max_count = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * d->n_bins));
  if (!L->col_start || !L->max_count ||
      cudaMemset(L->col_start, 0, sizeof(uint32_t) * (n_cols + 1)) != cudaSuccess) {
    lens_free(L);
    return nullptr;
  }
  return L;
}

// Columns from per-sample keys (kNoKey: skipped) and Earth pixels, with the
// per-column counts already accumulated in L->col_start: exclusive scan,
// scatter, canonical order inside each column, largest count per bin.
crp_status lens_columns(crp_lens* L, const uint32_t* key, const uint32_t* earth, uint64_t n) {
  uint32_t* fill = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * (L->n_cols + 1)));
  uint32_t* total = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t)));
  crp_status st = CRP_OK;
  if (!fill || !total) {
    st = CRP_E_OOM;
    set_error("lens: column workspace allocation failed");
  }
  if (st == CRP_OK) st = scan_inplace(L->col_start, L->n_cols + 1, total, nullptr);
  uint32_t n_entries = 0;
  if (st == CRP_OK) {
    cudaError_t e = cudaMemcpy(&n_entries, total, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(fill, L->col_start, sizeof(uint32_t) * (L->n_cols + 1),
                     cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) st = fail_cuda(e, "lens: counts");
  }
  if (st == CRP_OK) {
    L->n_entries = n_entries;
    L->entries = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * (n_entries ? n_entries : 1)));
    if (!L->entries) {
      st = CRP_E_OOM;
      set_error("lens: entries allocation failed");
    }
  }
  if (st == CRP_OK) {
    k_lens_scatter<<<blocks(n, 256), 256>>>(key, earth, n, fill, L->entries);
    k_lens_sort_columns<<<blocks(L->n_cols, 256), 256>>>(L->col_start, L->n_cols, L->entries);
    k_lens_max<<<L->n_bins, 256>>>(L->col_start, L->npix, L->n_bins, L->max_count);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = fail_cuda(e, "lens: columns");
  }
  dev_free(fill);
  dev_free(total);
  return st;
}

// Surrogate lens inputs and keys: x = (n, log10 R - 19) per sample; after the
// network, key = bin * npix + pixel(predicted border direction).
__global__ void k_surrogate_inputs(const double* dirs, const double* E, int64_t n, float* x) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    x[4 * k] = (float)dirs[3 * k];
    x[4 * k + 1] = (float)dirs[3 * k + 1];
    x[4 * k + 2] = (float)dirs[3 * k + 2];
    x[4 * k + 3] = (float)(log10(E[k]) - 19.0);
  }
}

__global__ void k_surrogate_keys(const double* dirs, const float* y, const int32_t* bin,
                                 int64_t n, int64_t nside, int64_t npix, uint32_t* key,
                                 uint32_t* earth, uint32_t* counts) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    earth[k] = (uint32_t)healpix_ring_pixel_guarded<false>(nside, dirs[3 * k], dirs[3 * k + 1],
                                                     dirs[3 * k + 2]);
    const int64_t j =
        healpix_ring_pixel_guarded<false>(nside, y[3 * k], y[3 * k + 1], y[3 * k + 2]);
    const uint32_t c = (uint32_t)((int64_t)bin[k] * npix + j);
    key[k] = c;
    atomicAdd(counts + c, 1u);
  }
}

}  // namespace

extern "C" {

crp_status crp_lens_build(crp_context* ctx, const crp_grid* galaxy, const crp_modules* m,
                          const crp_lens_desc* d, crp_lens** out, crp_stats* stats_out) {
  if (!ctx || !galaxy || !m || !d || !out || !d->dirs || !d->E || !d->bin) {
    set_error("crp_lens_build: NULL argument");
    return CRP_E_INVALID;
  }
  *out = nullptr;
  if (d->nside < 1 || d->nside > 8192 || d->n_bins < 1 || !(d->r_lo > 0.0) ||
      !(d->r_hi > d->r_lo) || d->n_samples < 1) {
    set_error("crp_lens_build: need 1 <= nside <= 8192, n_bins >= 1, 0 < r_lo < r_hi, samples");
    return CRP_E_INVALID;
  }
  const int64_t npix = 12ll * d->nside * d->nside;
  const int64_t n_cols = npix * d->n_bins;
  if (n_cols >= 0xFFFFFFFFll || d->n_samples >= 0xFFFFFFFFll) {
    set_error("crp_lens_build: too many columns or samples for 32-bit indices");
    return CRP_E_INVALID;
  }
  if (!(m->flags & CRP_BORDER)) {
    set_error("crp_lens_build: the modules must stop candidates at the border (CRP_BORDER)");
    return CRP_E_INVALID;
  }
  for (int64_t k = 0; k < d->n_samples; ++k) {
    if (d->bin[k] < 0 || d->bin[k] >= d->n_bins) {
      set_error("crp_lens_build: sample %lld has bin %d outside 0..%d", (long long)k, d->bin[k],
                d->n_bins - 1);
      return CRP_E_INVALID;
    }
  }
  DevState cst;
  uint64_t unused_n = 0, seed = 0;
  int device = 0;
  context_pool(ctx, &cst, &unused_n, &device, &seed);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);

  // back-track in a private pool so the caller's candidates stay untouched
  const uint64_t n = (uint64_t)d->n_samples;
  crp_context* bt = nullptr;
  crp_status st = crp_context_create(device, seed, n, &bt);
  std::vector<double> x(n, d->earth[0]), y(n, d->earth[1]), z(n, d->earth[2]);
  std::vector<double> ux(n), uy(n), uz(n);
  std::vector<int32_t> ones(n, 1), qneg(n, -1);
  for (uint64_t k = 0; k < n; ++k) {
    ux[k] = d->dirs[3 * k];
    uy[k] = d->dirs[3 * k + 1];
    uz[k] = d->dirs[3 * k + 2];
  }
  if (st == CRP_OK) {
    crp_candidate_arrays a;
    memset(&a, 0, sizeof(a));
    a.x = x.data(); a.y = y.data(); a.z = z.data();
    a.ux = ux.data(); a.uy = uy.data(); a.uz = uz.data();
    a.E = d->E;
    a.A = ones.data(); a.Z = ones.data(); a.q = qneg.data();
    st = crp_candidates_inject(bt, &a, n, 0, nullptr);
  }
  crp_stats bstats;
  memset(&bstats, 0, sizeof(bstats));
  if (st == CRP_OK) st = crp_propagate(bt, galaxy, m, nullptr, &bstats);
  if (stats_out) *stats_out = bstats;

  crp_lens* L = nullptr;
  uint32_t *key = nullptr, *earth = nullptr, *dbin = nullptr;
  if (st == CRP_OK) {
    key = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * n));
    earth = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * n));
    dbin = static_cast<uint32_t*>(dev_alloc(sizeof(int32_t) * n));
    if (!key || !earth || !dbin) {
      st = CRP_E_OOM;
      set_error("crp_lens_build: device allocation failed");
    }
  }
  if (st == CRP_OK) {
    DevState bst;
    uint64_t bn = 0, bseed = 0;
    int bdev = 0;
    context_pool(bt, &bst, &bn, &bdev, &bseed);
    L = lens_alloc(device, d, npix, n_cols);
    cudaError_t e = L ? cudaMemcpy(dbin, d->bin, sizeof(int32_t) * n, cudaMemcpyHostToDevice)
                      : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
      k_lens_keys<<<blocks(n, 256), 256>>>(bst, n, (const int32_t*)dbin, d->nside, npix, key,
                                           earth, L->col_start);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      st = L ? fail_cuda(e, "crp_lens_build: keys") : CRP_E_OOM;
      if (!L) set_error("crp_lens_build: device allocation failed");
    } else {
      st = lens_columns(L, key, earth, n);
    }
  }
  dev_free(key);
  dev_free(earth);
  dev_free(dbin);
  if (bt) crp_context_destroy(bt);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (st != CRP_OK) {
    lens_free(L);
    return st;
  }
  *out = L;
  return CRP_OK;
}

crp_status crp_lens_build_surrogate(crp_context* ctx, crp_mlp* mlp, const crp_lens_desc* d,
                                    crp_lens** out) {
  if (!ctx || !mlp || !d || !out || !d->dirs || !d->E || !d->bin) {
    set_error("crp_lens_build_surrogate: NULL argument");
    return CRP_E_INVALID;
  }
  *out = nullptr;
  if (d->nside < 1 || d->nside > 8192 || d->n_bins < 1 || !(d->r_lo > 0.0) ||
      !(d->r_hi > d->r_lo) || d->n_samples < 1) {
    set_error("crp_lens_build_surrogate: need 1 <= nside <= 8192, n_bins >= 1, 0 < r_lo < r_hi");
    return CRP_E_INVALID;
  }
  const int64_t npix = 12ll * d->nside * d->nside;
  const int64_t n_cols = npix * d->n_bins;
  if (n_cols >= 0xFFFFFFFFll || d->n_samples >= 0xFFFFFFFFll) {
    set_error("crp_lens_build_surrogate: too many columns or samples for 32-bit indices");
    return CRP_E_INVALID;
  }
  for (int64_t k = 0; k < d->n_samples; ++k) {
    if (d->bin[k] < 0 || d->bin[k] >= d->n_bins) {
      set_error("crp_lens_build_surrogate: sample %lld has bin %d outside 0..%d", (long long)k,
                d->bin[k], d->n_bins - 1);
      return CRP_E_INVALID;
    }
  }
  DevState cst;
  uint64_t unused_n = 0, seed = 0;
  int device = 0;
  context_pool(ctx, &cst, &unused_n, &device, &seed);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  const int64_t n = d->n_samples;
  const int64_t n_pad = (n + 127) / 128 * 128;
  double* ddirs = static_cast<double*>(dev_alloc(sizeof(double) * 3 * n));
  double* dE = static_cast<double*>(dev_alloc(sizeof(double) * n));
  int32_t* dbin = static_cast<int32_t*>(dev_alloc(sizeof(int32_t) * n));
  float* x = static_cast<float*>(dev_alloc(sizeof(float) * 4 * n_pad));
  float* y = static_cast<float*>(dev_alloc(sizeof(float) * 3 * n_pad));
  uint32_t* key = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * n));
  uint32_t* earth = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * n));
  crp_status st = CRP_OK;
  crp_lens* L = nullptr;
  if (!ddirs || !dE || !dbin || !x || !y || !key || !earth) {
    st = CRP_E_OOM;
    set_error("crp_lens_build_surrogate: device allocation failed");
  }
  if (st == CRP_OK) {
    cudaError_t e = cudaMemcpy(ddirs, d->dirs, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dE, d->E, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dbin, d->bin, sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(x, 0, sizeof(float) * 4 * n_pad);
    if (e == cudaSuccess) {
      k_surrogate_inputs<<<blocks(n, 256), 256>>>(ddirs, dE, n, x);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = fail_cuda(e, "crp_lens_build_surrogate: inputs");
  }
  if (st == CRP_OK) st = crp_mlp_forward(mlp, x, y, n_pad, nullptr);
  if (st == CRP_OK) {
    L = lens_alloc(device, d, npix, n_cols);
    if (!L) {
      st = CRP_E_OOM;
      set_error("crp_lens_build_surrogate: lens allocation failed");
    }
  }
  if (st == CRP_OK) {
    k_surrogate_keys<<<blocks(n, 256), 256>>>(ddirs, y, dbin, n, d->nside, npix, key, earth,
                                              L->col_start);
    const cudaError_t e = cudaGetLastError();
    st = e == cudaSuccess ? lens_columns(L, key, earth, (uint64_t)n)
                          : fail_cuda(e, "crp_lens_build_surrogate: keys");
  }
  dev_free(ddirs);
  dev_free(dE);
  dev_free(dbin);
  dev_free(x);
  dev_free(y);
  dev_free(key);
  dev_free(earth);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (st != CRP_OK) {
    lens_free(L);
    return st;
  }
  *out = L;
  return CRP_OK;
}

crp_status crp_lens_merge(const crp_lens* a, const crp_lens* b, const uint8_t* take_b,
                          crp_lens** out) {
  if (!a || !b || !take_b || !out) {
    set_error("crp_lens_merge: NULL argument");
    return CRP_E_INVALID;
  }
  if (a->device != b->device || a->nside != b->nside || a->n_bins != b->n_bins ||
      a->r_lo != b->r_lo || a->r_hi != b->r_hi) {
    set_error("crp_lens_merge: the lenses differ in device, nside, bins or rigidity range");
    return CRP_E_INVALID;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != a->device) {
    const cudaError_t e = cudaSetDevice(a->device);
    if (e != cudaSuccess) return fail_cuda(e, "crp_lens_merge: cudaSetDevice");
  }
  crp_status st = CRP_OK;
  const int64_t n_cols = a->n_cols, npix = a->npix;
  std::vector<uint32_t> ca(n_cols + 1), cb(n_cols + 1), cm(n_cols + 1), ma(a->n_bins),
      mb(a->n_bins), mm(a->n_bins);
  cudaError_t e = cudaMemcpy(ca.data(), a->col_start, 4 * (n_cols + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(cb.data(), b->col_start, 4 * (n_cols + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ma.data(), a->max_count, 4 * a->n_bins, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(mb.data(), b->max_count, 4 * a->n_bins, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) st = fail_cuda(e, "crp_lens_merge: copy in");
  // per bin: the chosen lens's columns (one contiguous range of its entries),
  // rebased onto the merged entry array
  uint64_t total = 0;
  if (st == CRP_OK) {
    for (int bin = 0; bin < a->n_bins; ++bin) {
      const std::vector<uint32_t>& c = take_b[bin] ? cb : ca;
      const int64_t c0 = (int64_t)bin * npix;
      for (int64_t j = 0; j < npix; ++j) cm[c0 + j] = (uint32_t)(total + (c[c0 + j] - c[c0]));
      total += c[c0 + npix] - c[c0];
      mm[bin] = take_b[bin] ? mb[bin] : ma[bin];
    }
    cm[n_cols] = (uint32_t)total;
    if (total > 0xffffffffull) {
      set_error("crp_lens_merge: more than 2^32 entries");
      st = CRP_E_INVALID;
    }
  }
  crp_lens* L = nullptr;
  if (st == CRP_OK) {
    crp_lens_desc d;
    memset(&d, 0, sizeof(d));
    d.nside = a->nside;
    d.n_bins = a->n_bins;
    d.r_lo = a->r_lo;
    d.r_hi = a->r_hi;
    L = lens_alloc(a->device, &d, npix, n_cols);
    if (L) {
      L->n_entries = (int64_t)total;
      L->entries = static_cast<uint32_t*>(dev_alloc(4 * (total ? total : 1)));
    }
    if (!L || !L->entries) {
      set_error("crp_lens_merge: allocation failed");
      st = CRP_E_OOM;
    }
  }
  if (st == CRP_OK) {
    e = cudaMemcpy(L->col_start, cm.data(), 4 * (n_cols + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(L->max_count, mm.data(), 4 * a->n_bins, cudaMemcpyHostToDevice);
    for (int bin = 0; bin < a->n_bins && e == cudaSuccess; ++bin) {
      const crp_lens* src = take_b[bin] ? b : a;
      const std::vector<uint32_t>& c = take_b[bin] ? cb : ca;
      const int64_t c0 = (int64_t)bin * npix;
      const uint32_t len = c[c0 + npix] - c[c0];
      if (len)
        e = cudaMemcpy(L->entries + cm[c0], src->entries + c[c0], 4 * (size_t)len,
                       cudaMemcpyDeviceToDevice);
    }
    if (e != cudaSuccess) st = fail_cuda(e, "crp_lens_merge: copy");
  }
  if (st != CRP_OK) {
    lens_free(L);
    L = nullptr;
  }
  if (prev >= 0 && prev != a->device) cudaSetDevice(prev);
  *out = L;
  return st;
}

crp_status crp_lens_destroy(crp_lens* L) {
  if (!L) return CRP_OK;
  cudaDeviceSynchronize();
  lens_free(L);
  return CRP_OK;
}

crp_status crp_lens_copy_out(const crp_lens* L, uint32_t* col_start, uint32_t* entries,
                             uint32_t* max_count, int64_t* n_entries) {
  if (!L || !n_entries) {
    set_error("crp_lens_copy_out: NULL argument");
    return CRP_E_INVALID;
  }
  *n_entries = L->n_entries;
  cudaError_t e = cudaSuccess;
  if (col_start)
    e = cudaMemcpy(col_start, L->col_start, sizeof(uint32_t) * (L->n_cols + 1),
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && entries && L->n_entries)
    e = cudaMemcpy(entries, L->entries, sizeof(uint32_t) * L->n_entries, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && max_count)
    e = cudaMemcpy(max_count, L->max_count, sizeof(uint32_t) * L->n_bins, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_lens_copy_out");
}

crp_status crp_lens_apply(crp_context* ctx, const crp_lens* L, int32_t what, void* stream) {
  if (!ctx || !L || what < CRP_COLLECT_ALL || what > CRP_COLLECT_AT_BORDER) {
    set_error("crp_lens_apply: bad argument");
    return CRP_E_INVALID;
  }
  DevState st;
  uint64_t n = 0, seed = 0;
  int device = 0;
  context_pool(ctx, &st, &n, &device, &seed);
  if (device != L->device) {
    set_error("crp_lens_apply: lens and context are on different devices");
    return CRP_E_INVALID;
  }
  if (n == 0) return CRP_OK;
  if (n >= (1ull << 31)) {
    set_error("crp_lens_apply: %llu candidates; at most 2^31 - 1", (unsigned long long)n);
    return CRP_E_INVALID;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double lg_lo = series_log(L->r_lo);
  const double inv = (double)L->n_bins / (series_log(L->r_hi) - lg_lo);
  // binary32 bin decisions need 1 / r_lo and inv_dlg as normal binary32 numbers
  const float inv_rlo_f = (float)(1.0 / L->r_lo), inv_f = (float)inv;
  const float inv2_f = (float)(inv * 0.693147180559945309417);
  const int use_f32 =
      std::isnormal(inv_rlo_f) && std::isnormal(inv_f) && std::isnormal(inv2_f) ? 1 : 0;
  LensArgs a;
  a.seed = seed;
  a.nside = L->nside;
  a.npix = L->npix;
  a.n_bins = L->n_bins;
  a.use_f32 = use_f32;
  a.lg_lo = lg_lo;
  a.inv_dlg = inv;
  a.inv_rlo_f = inv_rlo_f;
  a.inv_f = inv_f;
  a.inv2_f = inv2_f;
  a.col_start = L->col_start;
  a.entries = L->entries;
  a.max_count = L->max_count;
  uint32_t* list = nullptr;
  unsigned long long* cnt = nullptr;
  context_scratch(ctx, &list, &cnt);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    // 32 blocks of 256 per SM: several candidates per thread, so that the
    // next one's inputs load while this one is decided
    const uint64_t g = (uint64_t)(sms > 0 ? sms : 1) * 32;
    const uint64_t need = blocks(n, 256);
    const unsigned grid = (unsigned)(need < g ? need : g);
    const uint32_t n32 = (uint32_t)n;
    switch (what) {
      case CRP_COLLECT_ALL:
        k_lens_apply_f32<CRP_COLLECT_ALL><<<grid, 256, 0, s>>>(st, n32, a, list, cnt);
        break;
      case CRP_COLLECT_FINISHED:
        k_lens_apply_f32<CRP_COLLECT_FINISHED><<<grid, 256, 0, s>>>(st, n32, a, list, cnt);
        break;
      case CRP_COLLECT_DETECTED:
        k_lens_apply_f32<CRP_COLLECT_DETECTED><<<grid, 256, 0, s>>>(st, n32, a, list, cnt);
        break;
      case CRP_COLLECT_ACTIVE:
        k_lens_apply_f32<CRP_COLLECT_ACTIVE><<<grid, 256, 0, s>>>(st, n32, a, list, cnt);
        break;
      default:
        k_lens_apply_f32<CRP_COLLECT_AT_BORDER><<<grid, 256, 0, s>>>(st, n32, a, list, cnt);
        break;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_lens_apply_f64<<<(unsigned)(sms > 0 ? sms : 1) * 4, 256, 0, s>>>(st, a, list, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_lens_apply");
}

crp_status crp_histogram_healpix(crp_context* ctx, int32_t what, int32_t nside, int32_t source,
                                 uint64_t* out, void* stream) {
  if (!ctx || !out || nside < 1 || nside > 8192 || (source != 0 && source != 1) ||
      what < CRP_COLLECT_ALL || what > CRP_COLLECT_AT_BORDER) {
    set_error("crp_histogram_healpix: bad argument");
    return CRP_E_INVALID;
  }
  const uint64_t npix = 12ull * nside * nside;
  memset(out, 0, sizeof(uint64_t) * npix);
  DevState st;
  uint64_t n = 0, seed = 0;
  int device = 0;
  context_pool(ctx, &st, &n, &device, &seed);
  if (n == 0) return CRP_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* bins = static_cast<unsigned long long*>(dev_alloc(8 * npix));
  crp_status rc = CRP_OK;
  if (!bins) {
    set_error("crp_histogram_healpix: allocation failed");
    rc = CRP_E_OOM;
  } else {
    cudaError_t e = cudaMemsetAsync(bins, 0, 8 * npix, s);
    if (e == cudaSuccess) {
      k_hist_healpix<<<blocks(n, 256), 256, 0, s>>>(st, n, what, nside, source, bins);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, bins, 8 * npix, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail_cuda(e, "crp_histogram_healpix");
    dev_free(bins);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}


crp_status crp_histogram_healpix_device(crp_context* ctx, int32_t what, int32_t nside,
                                        int32_t source, uint64_t* out_dev, int32_t accumulate,
                                        void* stream) {
  if (!ctx || !out_dev || nside < 1 || nside > 8192 || (source != 0 && source != 1) ||
      what < CRP_COLLECT_ALL || what > CRP_COLLECT_AT_BORDER ||
      (reinterpret_cast<uintptr_t>(out_dev) & 7u)) {
    set_error("crp_histogram_healpix_device: bad argument");
    return CRP_E_INVALID;
  }
  const uint64_t npix = 12ull * nside * nside;
  DevState st;
  uint64_t n = 0, seed = 0;
  int device = 0;
  context_pool(ctx, &st, &n, &device, &seed);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) {
    const cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail_cuda(e, "crp_histogram_healpix_device: cudaSetDevice");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* bins = reinterpret_cast<unsigned long long*>(out_dev);
  cudaError_t e = cudaSuccess;
  if (!accumulate) e = cudaMemsetAsync(bins, 0, 8 * npix, s);
  if (e == cudaSuccess && n > 0) {
    k_hist_healpix<<<blocks(n, 256), 256, 0, s>>>(st, n, what, nside, source, bins);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_histogram_healpix_device");
}

}  // extern "C"
