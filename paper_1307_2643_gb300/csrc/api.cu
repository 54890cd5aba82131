// api.cu -- the C ABI: contexts, grids, tables, candidate pool, propagate
// driver and output collection.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>
#include <chrono>
#include <mutex>
#include <new>
#include <type_traits>
#include <utility>

#include "crp_internal.cuh"
#include "device_common.cuh"
#include "field_internal.h"

// ===========================================================================
// errors and memory
// ===========================================================================
namespace crp {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

crp_status fail_cuda(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  cudaGetLastError();  // clear a non-sticky error
  return CRP_E_CUDA;
}

static std::mutex g_alloc_mu;
static crp_alloc_fn g_alloc = nullptr;
static crp_free_fn g_free = nullptr;
static void* g_alloc_user = nullptr;

void* dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  crp_alloc_fn a;
  void* u;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
    u = g_alloc_user;
  }
  if (a) return a(bytes, u);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  crp_free_fn f;
  void* u;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f = g_free;
    u = g_alloc_user;
  }
  if (f)
    f(p, u);
  else
    cudaFree(p);
}

}  // namespace crp

using namespace crp;

// What a captured round-loop graph was built for (compared bytewise).
struct GraphKey {
  KParams kp;
  DevState st;
  const void* dc;
  int precision, block, variant, grid, sort_on, pad;
};

struct crp_context {
  int device;
  uint64_t seed;
  size_t capacity;
  size_t size;            // candidates in the pool
  void* pool;             // one allocation holding every SoA array
  DevState st;
  DevCounters* dc;        // device counters
  DevCounters* hc;        // pinned host mirror
  uint32_t* queue[2];     // work queues of the propagate rounds (capacity each)
  uint32_t* keys;         // spatial keys of the entries a round writes (capacity)
  uint32_t* bins;         // counting-sort histogram (kSortBins + 1)
  int sm_count;
  cudaEvent_t ev0, ev1;
  // graph mode: the round loop captured as one CUDA graph (while node)
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  GraphKey gkey;
  // the pool's arrays in layout order (checkpoint / restore walk this list)
  void* arr_ptr[64];
  uint32_t arr_elem[64];
  int n_arr;
};

struct crp_grid {
  crp_context* ctx;
  crp_grid_desc desc;
  void* nodes;
  void* cells;  // F32: per-cell corner records (8 float4 per cell), or null
  int64_t N;
};

struct crp_tables {
  crp_context* ctx;
  crp_tables_desc desc;
  double* data;   // beta | pion | gdr, n each
  float* data_f;  // binary32 copy of the three tables
  double* nuc;    // unstable nuclei (crp_tables_set_decay), or null
  int32_t nuc_amax;
};

namespace {

constexpr size_t kAlign = 256;
// Default slice: 2^20 accepted steps, i.e. a lane keeps its candidate to the
// end in practice (measured faster than requeueing every 512 steps: no
// round tails); a multiple of the mixed path's rebase period.
constexpr uint32_t kDefaultSlice = 1u << 20;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Lay out the SoA arrays of `cap` candidates inside one allocation; with a
// context, also list the arrays (pointer, element size) in layout order.
size_t layout_pool(char* base, size_t cap, DevState* st, crp_context* list = nullptr) {
  size_t off = 0;
  if (list) list->n_arr = 0;
  auto take = [&](auto** ptr, size_t elem) {
    using T = typename std::remove_pointer<typename std::remove_pointer<decltype(ptr)>::type>::type;
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "pool arrays hold 4- or 8-byte elements");
    if (base) *ptr = reinterpret_cast<T*>(base + off);
    if (base && list) {
      list->arr_ptr[list->n_arr] = base + off;
      list->arr_elem[list->n_arr] = (uint32_t)elem;
      ++list->n_arr;
    }
    off += align_up(elem * cap);
  };
  DevState s;
  memset(&s, 0, sizeof(s));
  take(&s.id, 8); take(&s.parent, 8);
  take(&s.x, 8); take(&s.y, 8); take(&s.z, 8);
  take(&s.ux, 8); take(&s.uy, 8); take(&s.uz, 8);
  take(&s.E, 8); take(&s.s, 8); take(&s.s_max, 8); take(&s.h, 8);
  take(&s.d_pion, 8); take(&s.d_pd, 8); take(&s.d_dec, 8);
  take(&s.x0, 8); take(&s.y0, 8); take(&s.z0, 8);
  take(&s.ux0, 8); take(&s.uy0, 8); take(&s.uz0, 8); take(&s.E0, 8);
  take(&s.n_acc, 8); take(&s.n_rej, 8);
  take(&s.A, 4); take(&s.Z, 4); take(&s.q, 4); take(&s.A0, 4); take(&s.Z0, 4); take(&s.status, 4);
  take(&s.draws, 4); take(&s.events, 4); take(&s.generation, 4); take(&s.n_pion, 4);
  take(&s.n_pd, 4); take(&s.n_dropped, 4); take(&s.flags, 4); take(&s.lens_pixel, 4);
  if (st) *st = s;
  return off;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

crp_status ensure_pool(crp_context* c) {
  if (c->pool) return CRP_OK;
  const size_t bytes = layout_pool(nullptr, c->capacity, nullptr);
  c->pool = dev_alloc(bytes);
  if (!c->pool) {
    set_error("candidate pool: cannot allocate %zu bytes for capacity %zu", bytes, c->capacity);
    return CRP_E_OOM;
  }
  layout_pool(static_cast<char*>(c->pool), c->capacity, &c->st, c);
  c->dc = static_cast<DevCounters*>(dev_alloc(sizeof(DevCounters)));
  c->queue[0] = static_cast<uint32_t*>(dev_alloc(c->capacity * sizeof(uint32_t)));
  c->queue[1] = static_cast<uint32_t*>(dev_alloc(c->capacity * sizeof(uint32_t)));
  c->keys = static_cast<uint32_t*>(dev_alloc(c->capacity * sizeof(uint32_t)));
  c->bins = static_cast<uint32_t*>(dev_alloc((kSortBins + 1) * sizeof(uint32_t)));
  if (!c->dc || !c->queue[0] || !c->queue[1] || !c->keys || !c->bins) {
    dev_free(c->pool);
    dev_free(c->dc);
    dev_free(c->queue[0]);
    dev_free(c->queue[1]);
    dev_free(c->keys);
    dev_free(c->bins);
    c->pool = nullptr;
    c->dc = nullptr;
    c->queue[0] = c->queue[1] = nullptr;
    c->keys = c->bins = nullptr;
    set_error("candidate pool: cannot allocate counters / work queues");
    return CRP_E_OOM;
  }
  return CRP_OK;
}

// ---------------------------------------------------------------------------
// inject kernels
// ---------------------------------------------------------------------------
__global__ void k_inject_init(DevState st, uint64_t base, uint64_t n, uint64_t first_id,
                              int has_id, int has_q, int has_smax, unsigned* bad) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + j;
    if (!has_id) st.id[i] = first_id + j;
    if (!has_q) st.q[i] = 1;
    if (!has_smax) st.s_max[i] = (double)INFINITY;
    const double ux = st.ux[i], uy = st.uy[i], uz = st.uz[i];
    const double un = ux * ux + uy * uy + uz * uz;
    const int A = st.A[i], Z = st.Z[i], q = st.q[i];
    const double E = st.E[i];
    const bool ok = A >= 1 && Z >= 0 && Z <= A && (q == 1 || q == -1) && E > 0.0 &&
                    E < (double)INFINITY && fabs(un - 1.0) < 1e-6 && st.s_max[i] >= 0.0;
    if (!ok) atomicAdd(bad, 1u);
    st.parent[i] = 0;
    st.x0[i] = st.x[i];
    st.y0[i] = st.y[i];
    st.z0[i] = st.z[i];
    st.ux0[i] = ux;
    st.uy0[i] = uy;
    st.uz0[i] = uz;
    st.E0[i] = E;
    st.A0[i] = A;
    st.Z0[i] = Z;
    st.s[i] = 0.0;
    st.h[i] = (double)INFINITY;  // first trial step: h_max
    st.d_pion[i] = 0.0;
    st.d_pd[i] = 0.0;
    st.d_dec[i] = 0.0;
    st.status[i] = CRP_ACTIVE;
    st.draws[i] = 0;
    st.events[i] = 0;
    st.generation[i] = 0;
    st.n_pion[i] = 0;
    st.n_pd[i] = 0;
    st.n_dropped[i] = 0;
    st.flags[i] = 0;
    st.lens_pixel[i] = 0xffffffffu;
    st.n_acc[i] = 0;
    st.n_rej[i] = 0;
  }
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

__global__ void k_to_float(const double* in, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// Work queue of the first round: every active candidate of the pool, with
// its spatial key.  The loop bound is warp-uniform so every lane takes part
// in each ballot.
__global__ void k_build_queue(DevState st, uint64_t n, FieldView f, int3 shift, int order,
                              uint32_t* queue, uint32_t* keys, unsigned long long* count) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int sh[3] = {shift.x, shift.y, shift.z};
  for (uint64_t base_i = blockIdx.x * (uint64_t)blockDim.x; base_i < n; base_i += stride) {
    const uint64_t i = base_i + threadIdx.x;
    const bool act = i < n && st.status[i] == CRP_ACTIVE;
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (act) {
      const uint64_t o = base + __popc(m & ((1u << lane) - 1u));
      queue[o] = (uint32_t)i;
      if (order != 1) {
        keys[o] = rigidity_key(st.E[i], st.Z[i]);
        continue;
      }
      const double r[3] = {st.x[i], st.y[i], st.z[i]};
      int cell[3];
      for (int d = 0; d < 3; ++d) {
        const double fl = floor((r[d] - f.origin[d]) * f.inv_spacing);
        int64_t c = (int64_t)fl % f.n[d];
        if (c < 0) c += f.n[d];
        cell[d] = (int)c;
      }
      keys[o] = brick_key(cell[0], cell[1], cell[2], sh);
    }
  }
}

// Counting sort of a work queue by its 15-bit keys (rigidity: lowest first;
// or spatial brick: lanes that run adjacent entries gather nearby cells).
__global__ void k_sort_hist(const uint32_t* keys, uint64_t n, uint32_t* bins) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(bins + keys[i], 1u);
}

__global__ void k_sort_scan(uint32_t* bins) {  // exclusive scan, one block of 1024
  __shared__ uint32_t part[1024];
  constexpr int per = kSortBins / 1024;
  const int t = threadIdx.x;
  uint32_t s = 0;
  for (int i = 0; i < per; ++i) s += bins[t * per + i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    uint32_t run = 0;
    for (int i = 0; i < 1024; ++i) {
      const uint32_t v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  uint32_t run = part[t];
  for (int i = 0; i < per; ++i) {
    const uint32_t v = bins[t * per + i];
    bins[t * per + i] = run;
    run += v;
  }
}

__global__ void k_sort_scatter(const uint32_t* keys, const uint32_t* in, uint64_t n,
                               uint32_t* bins, uint32_t* out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[atomicAdd(bins + keys[i], 1u)] = in[i];
}

__global__ void k_round_reset(DevCounters* dc) {
  dc->head = 0;
  dc->q_out = 0;
}

// ---- graph mode: the round loop with its queue length kept on the device ----
__device__ __forceinline__ uint64_t queued(const DevCounters* dc, uint64_t cap) {
  const unsigned long long q = dc->q_out;
  return q < cap ? q : cap;
}

__global__ void k_sort_hist_dev(const uint32_t* keys, const DevCounters* dc, uint64_t cap,
                                uint32_t* bins) {
  const uint64_t n = queued(dc, cap);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(bins + keys[i], 1u);
}

__global__ void k_sort_scatter_dev(const uint32_t* keys, const uint32_t* in,
                                   const DevCounters* dc, uint64_t cap, uint32_t* bins,
                                   uint32_t* out) {
  const uint64_t n = queued(dc, cap);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[atomicAdd(bins + keys[i], 1u)] = in[i];
}

__global__ void k_copy_queue_dev(const uint32_t* in, const DevCounters* dc, uint64_t cap,
                                 uint32_t* out) {
  const uint64_t n = queued(dc, cap);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// Start of a round: the previous round's output queue becomes this round's
// input; the loop ends (condition 0) when it is empty, when the step budget
// or deadline stopped the previous round, or after max_rounds rounds.
__global__ void k_graph_round(DevCounters* dc, uint64_t cap, cudaGraphConditionalHandle h,
                              unsigned long long max_rounds) {
  unsigned long long n = queued(dc, cap);
  dc->head = 0;
  dc->q_out = 0;
  bool go = n > 0 && dc->stop == 0;
  if (go && dc->rounds >= max_rounds) {
    dc->error_word |= ERR_ROUND_LIMIT;
    dc->stop = 1;
    go = false;
  }
  if (go)
    dc->rounds += 1;
  else
    n = 0;
  dc->n_in = n;
  if (!go) cudaGraphSetConditional(h, 0);
}

__global__ void k_count_active(const int32_t* status, uint64_t n, unsigned long long* out) {
  unsigned long long cnt = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    cnt += status[i] == CRP_ACTIVE;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// ---------------------------------------------------------------------------
// collect kernels: selection -> per-block counts -> scan -> ordered scatter
// ---------------------------------------------------------------------------
constexpr int kCollectBlock = 1024;

__device__ __forceinline__ bool selected(int what, int status) {
  switch (what) {
    case CRP_COLLECT_ALL: return true;
    case CRP_COLLECT_FINISHED: return status != CRP_ACTIVE;
    case CRP_COLLECT_DETECTED: return status == CRP_DETECTED;
    case CRP_COLLECT_ACTIVE: return status == CRP_ACTIVE;
    case CRP_COLLECT_AT_BORDER: return status == CRP_AT_BORDER;
  }
  return false;
}

__global__ void k_collect_count(const int32_t* status, uint64_t n, int what, unsigned* counts) {
  __shared__ unsigned sh;
  if (threadIdx.x == 0) sh = 0;
  __syncthreads();
  const uint64_t i = blockIdx.x * (uint64_t)kCollectBlock + threadIdx.x;
  const bool sel = i < n && selected(what, status[i]);
  const unsigned b = __ballot_sync(0xffffffffu, sel);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&sh, __popc(b));
  __syncthreads();
  if (threadIdx.x == 0) counts[blockIdx.x] = sh;
}

// exclusive scan of nb counts in a single block (fixed order)
__global__ void k_collect_scan(const unsigned* counts, int nb, unsigned long long* offsets) {
  __shared__ unsigned long long part[1024];
  const int t = threadIdx.x;
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = t * per, hi = min(nb, lo + per);
  unsigned long long s = 0;
  for (int i = lo; i < hi; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const unsigned long long v = part[i];
      part[i] = run;
      run += v;
    }
    offsets[nb] = run;
  }
  __syncthreads();
  unsigned long long run = part[t];
  for (int i = lo; i < hi; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
}

__global__ void k_collect_scatter(DevState st, uint64_t n, int what,
                                  const unsigned long long* offsets, crp_record* out) {
  __shared__ unsigned warp_base[kCollectBlock / 32];
  const uint64_t i = blockIdx.x * (uint64_t)kCollectBlock + threadIdx.x;
  const bool sel = i < n && selected(what, st.status[i]);
  const unsigned b = __ballot_sync(0xffffffffu, sel);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_base[warp] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int w = 0; w < kCollectBlock / 32; ++w) {
      const unsigned v = warp_base[w];
      warp_base[w] = run;
      run += v;
    }
  }
  __syncthreads();
  if (!sel) return;
  const uint64_t o = offsets[blockIdx.x] + warp_base[warp] + __popc(b & ((1u << lane) - 1u));
  crp_record r;
  r.id = st.id[i];
  r.parent_id = st.parent[i];
  r.x[0] = st.x[i]; r.x[1] = st.y[i]; r.x[2] = st.z[i];
  r.u[0] = st.ux[i]; r.u[1] = st.uy[i]; r.u[2] = st.uz[i];
  r.E = st.E[i];
  r.s = st.s[i];
  r.x0[0] = st.x0[i]; r.x0[1] = st.y0[i]; r.x0[2] = st.z0[i];
  r.u0[0] = st.ux0[i]; r.u0[1] = st.uy0[i]; r.u0[2] = st.uz0[i];
  r.E0 = st.E0[i];
  r.s_max = st.s_max[i];
  r.n_acc = st.n_acc[i];
  r.n_rej = st.n_rej[i];
  r.A = st.A[i]; r.Z = st.Z[i]; r.A0 = st.A0[i]; r.Z0 = st.Z0[i]; r.q = st.q[i];
  r.status = st.status[i];
  r.n_pion = st.n_pion[i];
  r.n_pd = st.n_pd[i];
  r.draws = st.draws[i];
  r.generation = st.generation[i];
  r.n_dropped = st.n_dropped[i];
  r.lens_pixel = st.lens_pixel[i];
  out[o] = r;
}

__global__ void k_hist_energy(const int32_t* status, const double* E, uint64_t n, int what,
                              double l0, double inv_dl, int nb, unsigned long long* bins) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (!selected(what, status[i])) continue;
    const double t = (log(E[i]) - l0) * inv_dl;
    if (!(t >= 0.0) || t >= (double)nb) continue;
    atomicAdd(bins + (int)t, 1ull);
  }
}

int blocks_for(uint64_t n, int block) {
  const uint64_t b = (n + block - 1) / block;
  return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* crp_last_error(void) { return g_err; }

int32_t crp_version(void) { return 100; }

crp_status crp_set_allocator(crp_alloc_fn alloc, crp_free_fn release, void* user) {
  if ((alloc == nullptr) != (release == nullptr)) {
    set_error("crp_set_allocator: alloc and release must both be set or both be NULL");
    return CRP_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = release;
  g_alloc_user = user;
  return CRP_OK;
}

crp_status crp_context_create(int32_t device, uint64_t seed, size_t capacity, crp_context** out) {
  if (!out || capacity == 0) {
    set_error("crp_context_create: out must be non-NULL and capacity > 0");
    return CRP_E_INVALID;
  }
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail_cuda(e, "crp_context_create: cudaGetDeviceCount");
  if (device < 0 || device >= ndev) {
    set_error("crp_context_create: device %d not present (%d devices)", device, ndev);
    return CRP_E_INVALID;
  }
  DeviceGuard g(device);
  crp_context* c = new (std::nothrow) crp_context;
  if (!c) {
    set_error("crp_context_create: host allocation failed");
    return CRP_E_OOM;
  }
  memset(c, 0, sizeof(*c));
  c->device = device;
  c->seed = seed;
  c->capacity = capacity;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  e = cudaMallocHost(&c->hc, sizeof(DevCounters));
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e != cudaSuccess) {
    delete c;
    return fail_cuda(e, "crp_context_create");
  }
  *out = c;
  return CRP_OK;
}

crp_status crp_context_destroy(crp_context* c) {
  if (!c) return CRP_OK;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  dev_free(c->pool);
  dev_free(c->dc);
  dev_free(c->queue[0]);
  dev_free(c->queue[1]);
  dev_free(c->keys);
  dev_free(c->bins);
  if (c->hc) cudaFreeHost(c->hc);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return CRP_OK;
}

crp_status crp_context_size(const crp_context* c, size_t* n_out) {
  if (!c || !n_out) {
    set_error("crp_context_size: NULL argument");
    return CRP_E_INVALID;
  }
  *n_out = c->size;
  return CRP_OK;
}

// ---------------------------------------------------------------------------
crp_status crp_grid_create(crp_context* c, const crp_grid_desc* d, crp_grid** out) {
  if (!c || !d || !out) {
    set_error("crp_grid_create: NULL argument");
    return CRP_E_INVALID;
  }
  *out = nullptr;
  if (d->n[0] < 2 || d->n[1] < 2 || d->n[2] < 2 || !(d->spacing > 0.0) ||
      (d->dtype != CRP_F32 && d->dtype != CRP_F64)) {
    set_error("crp_grid_create: need n >= 2 per axis, spacing > 0, dtype F32|F64");
    return CRP_E_INVALID;
  }
  if (d->n[0] > (1 << 20) || d->n[1] > (1 << 20) || d->n[2] > (1 << 20)) {
    set_error("crp_grid_create: at most 2^20 nodes per axis");
    return CRP_E_INVALID;
  }
  if (d->cell_records != 0 && d->cell_records != -1) {
    set_error("crp_grid_create: cell_records must be 0 or -1");
    return CRP_E_INVALID;
  }
  const int64_t N = d->n[0] * d->n[1] * d->n[2];
  if (d->source == CRP_GRID_TURBULENT) {
    if (!(d->lmin > 0.0) || !(d->lmax >= d->lmin) || !(d->brms >= 0.0)) {
      set_error("crp_grid_create: turbulence needs 0 < lmin <= lmax and brms >= 0");
      return CRP_E_INVALID;
    }
  } else if (d->source == CRP_GRID_FROM_HOST || d->source == CRP_GRID_FROM_DEVICE) {
    if (!d->data || (d->data_dtype != CRP_F32 && d->data_dtype != CRP_F64)) {
      set_error("crp_grid_create: data pointer and data_dtype F32|F64 required");
      return CRP_E_INVALID;
    }
  } else {
    set_error("crp_grid_create: unknown source %d", d->source);
    return CRP_E_INVALID;
  }
  DeviceGuard g(c->device);
  crp_grid* gr = new (std::nothrow) crp_grid;
  if (!gr) {
    set_error("crp_grid_create: host allocation failed");
    return CRP_E_OOM;
  }
  gr->ctx = c;
  gr->desc = *d;
  gr->desc.data = nullptr;
  gr->N = N;
  gr->nodes = dev_alloc((size_t)N * node_bytes(d->dtype));
  if (!gr->nodes) {
    delete gr;
    set_error("crp_grid_create: cannot allocate %zu bytes", (size_t)N * node_bytes(d->dtype));
    return CRP_E_OOM;
  }
  crp_status st = CRP_OK;
  cudaStream_t s = 0;
  if (d->source == CRP_GRID_TURBULENT) {
    st = grid_turbulence(d, gr->nodes, s);
  } else {
    const size_t esz = d->data_dtype == CRP_F32 ? 4 : 8;
    const size_t bytes = (size_t)N * 3 * esz;
    const void* src = d->data;
    void* staging = nullptr;
    if (d->source == CRP_GRID_FROM_HOST) {
      staging = dev_alloc(bytes);
      if (!staging) {
        st = CRP_E_OOM;
        set_error("crp_grid_create: cannot allocate staging buffer");
      } else {
        cudaError_t e = cudaMemcpy(staging, d->data, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = fail_cuda(e, "crp_grid_create: copy from host");
        src = staging;
      }
    }
    if (st == CRP_OK) st = grid_pack(src, d->data_dtype, N, d->dtype, gr->nodes, s);
    if (st == CRP_OK) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = fail_cuda(e, "crp_grid_create");
    }
    dev_free(staging);
  }
  gr->cells = nullptr;
  if (st == CRP_OK && d->dtype == CRP_F32 && d->cell_records == 0 && N < (int64_t(1) << 32)) {
    // optional: a grid without records still works (node gathers); records
    // are indexed in 32 bits by some kernels, so only below 2^32 cells
    gr->cells = dev_alloc((size_t)N * 8 * sizeof(float4));
    if (gr->cells) {
      st = grid_cells(gr->nodes, d->n, gr->cells, s);
      if (st == CRP_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fail_cuda(e, "crp_grid_create: cell records");
      }
    }
  }
  if (st != CRP_OK) {
    dev_free(gr->cells);
    dev_free(gr->nodes);
    delete gr;
    return st;
  }
  *out = gr;
  return CRP_OK;
}

crp_status crp_grid_destroy(crp_grid* g) {
  if (!g) return CRP_OK;
  DeviceGuard dg(g->ctx->device);
  cudaDeviceSynchronize();
  dev_free(g->cells);
  dev_free(g->nodes);
  delete g;
  return CRP_OK;
}

crp_status crp_grid_copy_out(const crp_grid* g, double* host_out) {
  if (!g || !host_out) {
    set_error("crp_grid_copy_out: NULL argument");
    return CRP_E_INVALID;
  }
  DeviceGuard dg(g->ctx->device);
  const size_t bytes = (size_t)g->N * 3 * sizeof(double);
  double* tmp = static_cast<double*>(dev_alloc(bytes));
  if (!tmp) {
    set_error("crp_grid_copy_out: cannot allocate %zu bytes", bytes);
    return CRP_E_OOM;
  }
  crp_status st = grid_unpack(g->nodes, g->desc.dtype, g->N, tmp, 0);
  if (st == CRP_OK) {
    cudaError_t e = cudaMemcpy(host_out, tmp, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = fail_cuda(e, "crp_grid_copy_out");
  }
  dev_free(tmp);
  return st;
}

// ---------------------------------------------------------------------------
static crp_status tables_check(const crp_tables_desc* d) {
  if (!d || d->n < 2 || d->n > (1 << 24) || !(d->gamma_lo > 0.0) || !(d->gamma_hi > d->gamma_lo) ||
      !(d->length_unit_m > 0.0)) {
    set_error("tables: need n >= 2, 0 < gamma_lo < gamma_hi, length_unit_m > 0");
    return CRP_E_INVALID;
  }
  for (int k = 0; k < 2; ++k) {
    if (!(d->irb_dilution[k] >= 0.0) || (d->irb_dilution[k] > 0.0 && !(d->irb_T_K[k] > 0.0))) {
      set_error("tables: background component %d needs dilution >= 0 and T > 0", k);
      return CRP_E_INVALID;
    }
  }
  return CRP_OK;
}

static crp_tables* tables_alloc(crp_context* c, const crp_tables_desc* d) {
  crp_tables* t = new (std::nothrow) crp_tables;
  if (!t) return nullptr;
  t->ctx = c;
  t->desc = *d;
  t->nuc = nullptr;
  t->nuc_amax = 0;
  t->data = static_cast<double*>(dev_alloc(3 * (size_t)d->n * sizeof(double)));
  t->data_f = static_cast<float*>(dev_alloc(3 * (size_t)d->n * sizeof(float)));
  if (!t->data || !t->data_f) {
    dev_free(t->data);
    dev_free(t->data_f);
    delete t;
    return nullptr;
  }
  return t;
}

crp_status crp_tables_build(crp_context* c, const crp_tables_desc* d, crp_tables** out) {
  if (!c || !out) {
    set_error("crp_tables_build: NULL argument");
    return CRP_E_INVALID;
  }
  if (tables_check(d) != CRP_OK) return CRP_E_INVALID;
  if (!(d->T_cmb > 0.0) || !(d->gdr_fwhm_eV > 0.0) || !(d->gdr_hi_eV > d->gdr_lo_eV)) {
    set_error("crp_tables_build: need T_cmb > 0, gdr_fwhm > 0, gdr_lo < gdr_hi");
    return CRP_E_INVALID;
  }
  DeviceGuard g(c->device);
  crp_tables* t = tables_alloc(c, d);
  if (!t) {
    set_error("crp_tables_build: allocation failed");
    return CRP_E_OOM;
  }
  crp_status st = tables_compute(d, t->data, t->data + d->n, t->data + 2 * d->n, 0);
  if (st == CRP_OK) {
    k_to_float<<<blocks_for(3 * d->n, 256), 256>>>(t->data, t->data_f, 3 * d->n);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = fail_cuda(e, "crp_tables_build: float copy");
  }
  if (st != CRP_OK) {
    dev_free(t->data);
    dev_free(t->data_f);
    delete t;
    return st;
  }
  *out = t;
  return CRP_OK;
}

crp_status crp_tables_from_host(crp_context* c, const crp_tables_desc* d, const double* beta,
                                const double* pion, const double* gdr, crp_tables** out) {
  if (!c || !out || !beta || !pion || !gdr) {
    set_error("crp_tables_from_host: NULL argument");
    return CRP_E_INVALID;
  }
  if (tables_check(d) != CRP_OK) return CRP_E_INVALID;
  DeviceGuard g(c->device);
  crp_tables* t = tables_alloc(c, d);
  if (!t) {
    set_error("crp_tables_from_host: allocation failed");
    return CRP_E_OOM;
  }
  const size_t b = (size_t)d->n * sizeof(double);
  cudaError_t e = cudaMemcpy(t->data, beta, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->data + d->n, pion, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->data + 2 * d->n, gdr, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_to_float<<<blocks_for(3 * d->n, 256), 256>>>(t->data, t->data_f, 3 * d->n);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    dev_free(t->data);
    dev_free(t->data_f);
    delete t;
    return fail_cuda(e, "crp_tables_from_host");
  }
  *out = t;
  return CRP_OK;
}

crp_status crp_tables_copy_out(const crp_tables* t, double* beta, double* pion, double* gdr) {
  if (!t || !beta || !pion || !gdr) {
    set_error("crp_tables_copy_out: NULL argument");
    return CRP_E_INVALID;
  }
  DeviceGuard g(t->ctx->device);
  const size_t b = (size_t)t->desc.n * sizeof(double);
  cudaError_t e = cudaMemcpy(beta, t->data, b, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(pion, t->data + t->desc.n, b, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(gdr, t->data + 2 * t->desc.n, b, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_tables_copy_out");
}

crp_status crp_tables_destroy(crp_tables* t) {
  if (!t) return CRP_OK;
  DeviceGuard g(t->ctx->device);
  cudaDeviceSynchronize();
  dev_free(t->data);
  dev_free(t->data_f);
  dev_free(t->nuc);
  delete t;
  return CRP_OK;
}

crp_status crp_tables_set_decay(crp_tables* t, int64_t n, const int32_t* A, const int32_t* Z,
                                const double* tau_s, const double* branching) {
  if (!t || n < 0 || (n > 0 && (!A || !Z || !tau_s || !branching))) {
    set_error("crp_tables_set_decay: bad argument");
    return CRP_E_INVALID;
  }
  int32_t amax = 2;
  for (int64_t i = 0; i < n; ++i) {
    const int a = A[i], z = Z[i];
    if (a < 2 || a > CRP_DECAY_MAX_A || z < 1 || z > a - 1) {
      set_error("crp_tables_set_decay: entry %lld: (A, Z) = (%d, %d) outside 2 <= A <= %d, "
                "1 <= Z <= A - 1", (long long)i, a, z, CRP_DECAY_MAX_A);
      return CRP_E_INVALID;
    }
    if (!(tau_s[i] > 0.0)) {
      set_error("crp_tables_set_decay: entry %lld: lifetime %g must be > 0", (long long)i,
                tau_s[i]);
      return CRP_E_INVALID;
    }
    const double* b = branching + 4 * i;
    double sum = 0.0;
    // daughters of beta-, beta+, neutron emission, proton emission
    const int da[4] = {a, a, a - 1, a - 1}, dz[4] = {z + 1, z - 1, z, z - 1};
    for (int k = 0; k < 4; ++k) {
      if (!(b[k] >= 0.0) || !std::isfinite(b[k])) {
        set_error("crp_tables_set_decay: entry %lld: branching fraction %d is %g", (long long)i,
                  k, b[k]);
        return CRP_E_INVALID;
      }
      if (b[k] > 0.0 && da[k] >= 2 && (dz[k] < 1 || dz[k] > da[k] - 1)) {
        set_error("crp_tables_set_decay: entry %lld: channel %d of (%d, %d) would make (%d, %d)",
                  (long long)i, k, a, z, da[k], dz[k]);
        return CRP_E_INVALID;
      }
      sum += b[k];
    }
    if (!(fabs(sum - 1.0) <= 1e-9)) {
      set_error("crp_tables_set_decay: entry %lld: branching fractions sum to %.17g", (long long)i,
                sum);
      return CRP_E_INVALID;
    }
    if (a > amax) amax = a;
  }
  const int64_t slots = (int64_t)(amax + 1) * (amax + 2) / 2;
  std::vector<double> h((size_t)(slots * kNucEntry), 0.0);
  std::vector<char> seen((size_t)slots, 0);
  for (int64_t k = 0; k < slots; ++k) h[(size_t)(k * kNucEntry)] = (double)INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t k = (int64_t)A[i] * (A[i] + 1) / 2 + Z[i];
    if (seen[(size_t)k]) {
      set_error("crp_tables_set_decay: (A, Z) = (%d, %d) listed twice", A[i], Z[i]);
      return CRP_E_INVALID;
    }
    seen[(size_t)k] = 1;
    const double* b = branching + 4 * i;
    double* e = h.data() + k * kNucEntry;
    // cumulative fractions, summed left to right
    const double c1 = b[0], c2 = c1 + b[1], c3 = c2 + b[2];
    int past = 3;
    if (!(b[3] > 0.0)) past = b[2] > 0.0 ? 2 : (b[1] > 0.0 ? 1 : 0);
    e[0] = tau_s[i];
    e[1] = c1;
    e[2] = c2;
    e[3] = c3;
    e[4] = (double)past;
  }
  DeviceGuard g(t->ctx->device);
  double* d = nullptr;
  if (n > 0) {
    d = static_cast<double*>(dev_alloc(h.size() * sizeof(double)));
    if (!d) {
      set_error("crp_tables_set_decay: allocation failed");
      return CRP_E_OOM;
    }
    const cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(double),
                                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      dev_free(d);
      return fail_cuda(e, "crp_tables_set_decay");
    }
  }
  cudaDeviceSynchronize();
  dev_free(t->nuc);
  t->nuc = d;
  t->nuc_amax = n > 0 ? amax : 0;
  return CRP_OK;
}

// ---------------------------------------------------------------------------
crp_status crp_candidates_inject(crp_context* c, const crp_candidate_arrays* a, size_t n,
                                 uint64_t first_id, void* stream) {
  if (!c || !a) {
    set_error("crp_candidates_inject: NULL argument");
    return CRP_E_INVALID;
  }
  if (n == 0) return CRP_OK;
  if (!a->x || !a->y || !a->z || !a->ux || !a->uy || !a->uz || !a->E || !a->A || !a->Z) {
    set_error("crp_candidates_inject: x, y, z, ux, uy, uz, E, A, Z are required");
    return CRP_E_INVALID;
  }
  if (n > c->capacity - c->size) {
    set_error("crp_candidates_inject: %zu candidates do not fit (pool %zu of %zu used)", n,
              c->size, c->capacity);
    return CRP_E_QUEUE_FULL;
  }
  DeviceGuard g(c->device);
  crp_status st = ensure_pool(c);
  if (st != CRP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind kind = a->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t base = c->size;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t elem) {
    if (e == cudaSuccess && src) e = cudaMemcpyAsync(dst, src, n * elem, kind, s);
  };
  cp(c->st.x + base, a->x, 8);
  cp(c->st.y + base, a->y, 8);
  cp(c->st.z + base, a->z, 8);
  cp(c->st.ux + base, a->ux, 8);
  cp(c->st.uy + base, a->uy, 8);
  cp(c->st.uz + base, a->uz, 8);
  cp(c->st.E + base, a->E, 8);
  cp(c->st.A + base, a->A, 4);
  cp(c->st.Z + base, a->Z, 4);
  cp(c->st.q + base, a->q, 4);
  cp(c->st.s_max + base, a->s_max, 8);
  cp(c->st.id + base, a->id, 8);
  if (e != cudaSuccess) return fail_cuda(e, "crp_candidates_inject: copy");
  e = cudaMemsetAsync(&c->dc->error_word, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return fail_cuda(e, "crp_candidates_inject: memset");
  k_inject_init<<<blocks_for(n, 256), 256, 0, s>>>(c->st, base, n, first_id, a->id != nullptr,
                                                     a->q != nullptr, a->s_max != nullptr,
                                                     &c->dc->error_word);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&c->hc->error_word, &c->dc->error_word, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "crp_candidates_inject");
  if (c->hc->error_word) {
    set_error("crp_candidates_inject: %u invalid candidates (need A >= 1, 0 <= Z <= A, q = +-1, "
              "finite E > 0, |u| = 1, s_max >= 0); nothing injected",
              c->hc->error_word);
    return CRP_E_INVALID;
  }
  c->size += n;
  return CRP_OK;
}

crp_status crp_candidates_clear(crp_context* c) {
  if (!c) {
    set_error("crp_candidates_clear: NULL argument");
    return CRP_E_INVALID;
  }
  c->size = 0;
  return CRP_OK;
}

// ---------------------------------------------------------------------------
static void fill_field_view(const crp_grid* g, FieldView& f) {
  f.data = g->nodes;
  f.cells = static_cast<const float4*>(g->cells);
  f.cache_ok = g->N < 0xffffffffll ? 1 : 0;
  for (int d = 0; d < 3; ++d) {
    f.n[d] = g->desc.n[d];
    f.mask[d] = (g->desc.n[d] & (g->desc.n[d] - 1)) == 0 ? g->desc.n[d] - 1 : -1;
    f.origin[d] = g->desc.origin[d];
  }
  f.spacing = g->desc.spacing;
  f.inv_spacing = 1.0 / g->desc.spacing;
  f.inv_spacing_f = (float)f.inv_spacing;
  f.dtype = g->desc.dtype;
}

// Galactic-field parameters: binary64 values first, then the binary32
// copies the mixed path uses.
static void fill_galactic(const crp_modules* m, KParams& kp) {
  for (int d = 0; d < 3; ++d) kp.gal_c[d] = m->gal_center[d];
  kp.disk_b = m->disk_b;
  kp.sin_pitch = sin(m->disk_pitch_rad);
  kp.cos_pitch = cos(m->disk_pitch_rad);
  kp.disk_hz = m->disk_hz;
  kp.disk_rmin = m->disk_rmin;
  kp.disk_rmax = m->disk_rmax;
  kp.halo_b = m->halo_b;
  kp.halo_z0 = m->halo_z0;
  kp.halo_sigma = m->halo_sigma;
  kp.gdisk_b = (float)kp.disk_b;
  kp.gsin = (float)kp.sin_pitch;
  kp.gcos = (float)kp.cos_pitch;
  kp.ginv_hz = kp.disk_hz > 0.0 ? (float)(1.0 / kp.disk_hz) : 0.f;
  kp.grmin = (float)kp.disk_rmin;
  kp.grmax = (float)kp.disk_rmax;
  kp.ghalo_b = (float)kp.halo_b;
  kp.ghalo_z0 = (float)kp.halo_z0;
  kp.ghalo_inv2s2 =
      kp.halo_sigma > 0.0 ? (float)(1.0 / (2.0 * kp.halo_sigma * kp.halo_sigma)) : 0.f;
}

// Multi-arm galactic field: validate m->gmf and convert it.  Each binary64
// constant is the single expression the model's statement gives (so the
// binary64 field is reproducible); binary32 copies and reciprocals follow.
static crp_status fill_gmf(const crp_modules* m, KParams& kp, const char* who) {
  memset(&kp.gm, 0, sizeof(kp.gm));
  if (!(m->flags & CRP_GMF)) return CRP_OK;
  const crp_gmf* g = m->gmf;
  if (!g) {
    set_error("%s: CRP_GMF without m->gmf", who);
    return CRP_E_INVALID;
  }
  const double tan_p = tan(g->pitch_rad);
  const double period = 2.0 * M_PI * tan_p;
  bool ok = fabs(g->pitch_rad) > 0.0 && fabs(g->pitch_rad) < 0.5 * M_PI && g->arm_rx[0] > 0.0 &&
            g->w_disk > 0.0 && g->halo_wh > 0.0 && g->halo_z0 > 0.0 && g->r_in > 0.0 &&
            g->r_cut_in >= 0.0 && g->r_cut_out >= 0.0;
  for (int j = 1; j < 8 && ok; ++j) ok = g->arm_rx[j] > g->arm_rx[j - 1];
  ok = ok && tan_p > 0.0 && log(g->arm_rx[7]) - log(g->arm_rx[0]) < period;
  if (ok && g->x_b != 0.0)
    ok = g->x_theta_rad > 0.0 && g->x_theta_rad < 0.5 * M_PI && g->x_rc > 0.0 && g->x_r > 0.0;
  for (int j = 0; j < 8 && ok; ++j) ok = std::isfinite(g->arm_b[j]);
  if (!ok) {
    set_error("%s: invalid crp_gmf (arm radii ascending within one spiral turn, "
              "0 < pitch < pi/2, positive widths, scales and X-field geometry)", who);
    return CRP_E_INVALID;
  }
  GmfView& v = kp.gm;
  v.ln_r0 = log(g->arm_rx[0]);
  for (int j = 0; j < 8; ++j) {
    v.arm_b[j] = g->arm_b[j];
    v.d_arm[j] = log(g->arm_rx[j]) - v.ln_r0;
  }
  v.tan_p = tan_p;
  v.sin_p = sin(g->pitch_rad);
  v.cos_p = cos(g->pitch_rad);
  v.period = period;
  v.ring_b = g->ring_b;
  v.r_ring = g->r_ring;
  v.r_in = g->r_in;
  v.r_out = g->r_out;
  v.h_disk = g->h_disk;
  v.w_disk = g->w_disk;
  v.halo_bn = g->halo_bn;
  v.halo_bs = g->halo_bs;
  v.halo_rn = g->halo_rn;
  v.halo_rs = g->halo_rs;
  v.halo_wh = g->halo_wh;
  v.halo_z0 = g->halo_z0;
  v.x_b = g->x_b;
  v.tan_t = g->x_b != 0.0 ? tan(g->x_theta_rad) : 1.0;
  v.sin_t = sin(g->x_theta_rad);
  v.cos_t = cos(g->x_theta_rad);
  v.x_rc = g->x_rc;
  v.x_r = g->x_r;
  v.cut_in2 = g->r_cut_in * g->r_cut_in;
  v.cut_out2 = g->r_cut_out * g->r_cut_out;
  for (int j = 0; j < 8; ++j) {
    v.f_arm_b[j] = (float)v.arm_b[j];
    v.f_d_arm[j] = (float)v.d_arm[j];
  }
  v.f_ln_r0 = (float)v.ln_r0;
  v.f_tan_p = (float)tan_p;
  v.f_sin_p = (float)v.sin_p;
  v.f_cos_p = (float)v.cos_p;
  v.f_period = (float)period;
  v.f_inv_period = (float)(1.0 / period);
  v.f_ring_b = (float)v.ring_b;
  v.f_r_ring = (float)v.r_ring;
  v.f_r_in = (float)v.r_in;
  v.f_r_out = (float)v.r_out;
  v.f_h_disk = (float)v.h_disk;
  v.f_m2_inv_w_disk = (float)(-2.0 / v.w_disk);
  v.f_halo_bn = (float)v.halo_bn;
  v.f_halo_bs = (float)v.halo_bs;
  v.f_halo_rn = (float)v.halo_rn;
  v.f_halo_rs = (float)v.halo_rs;
  v.f_m2_inv_halo_wh = (float)(-2.0 / v.halo_wh);
  v.f_inv_halo_z0 = (float)(1.0 / v.halo_z0);
  v.f_x_b = (float)v.x_b;
  v.f_inv_tan_t = (float)(1.0 / v.tan_t);
  v.f_sin_t = (float)v.sin_t;
  v.f_cos_t = (float)v.cos_t;
  v.f_x_rc = (float)v.x_rc;
  v.f_inv_x_r = v.x_r > 0.0 ? (float)(1.0 / v.x_r) : 0.f;
  v.f_q = (float)(v.x_rc * v.tan_t);
  v.f_cut_in2 = (float)v.cut_in2;
  v.f_cut_out2 = (float)v.cut_out2;
  return CRP_OK;
}

// Graph mode: capture the round loop once (a while node whose body sorts
// the queue, starts the round and runs the propagate kernel; the loop
// condition is set on the device) and replay it; rebuilt when the launch
// parameters change.  One graph launch replaces a host round trip per round.
static cudaError_t graph_rounds(crp_context* c, const KParams& kp, int precision, int block,
                                int variant, int grid, bool sort_on, cudaStream_t s,
                                float* ms_out) {
  GraphKey key;
  memset(&key, 0, sizeof(key));
  key.kp = kp;
  key.st = c->st;
  key.dc = c->dc;
  key.precision = precision;
  key.block = block;
  key.variant = variant;
  key.grid = grid;
  key.sort_on = sort_on ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (!c->gexec || memcmp(&key, &c->gkey, sizeof(key)) != 0) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&c->graph, 0);
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess)
      e = cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault);
    // the parameter union has no usable default constructor: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char np_mem[sizeof(cudaGraphNodeParams)];
    memset(np_mem, 0, sizeof(np_mem));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_mem);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      cudaStream_t cs = c->cap_stream;
      e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        const int gb = c->sm_count * 8;
        const uint64_t cap = c->capacity;
        if (sort_on) {
          cudaMemsetAsync(c->bins, 0, (kSortBins + 1) * sizeof(uint32_t), cs);
          k_sort_hist_dev<<<gb, 256, 0, cs>>>(c->keys, c->dc, cap, c->bins);
          k_sort_scan<<<1, 1024, 0, cs>>>(c->bins);
          k_sort_scatter_dev<<<gb, 256, 0, cs>>>(c->keys, c->queue[1], c->dc, cap, c->bins,
                                                 c->queue[0]);
        } else {
          k_copy_queue_dev<<<gb, 256, 0, cs>>>(c->queue[1], c->dc, cap, c->queue[0]);
        }
        k_graph_round<<<1, 1, 0, cs>>>(c->dc, cap, h, 1ull << 20);
        e = precision == CRP_FP64
                ? launch_propagate_fp64(kp, c->st, c->dc, grid, block, cs)
                : launch_propagate_mixed(kp, c->st, c->dc, grid, block, variant, cs);
        cudaGraph_t done = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &done);
        if (e == cudaSuccess) e = e2;
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, c->graph, 0);
    if (e != cudaSuccess) {
      if (c->gexec) cudaGraphExecDestroy(c->gexec);
      if (c->graph) cudaGraphDestroy(c->graph);
      c->gexec = nullptr;
      c->graph = nullptr;
      return e;
    }
    c->gkey = key;
  }
  cudaEventRecord(c->ev0, s);
  e = cudaGraphLaunch(c->gexec, s);
  cudaEventRecord(c->ev1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  *ms_out = ms;
  return e;
}

crp_status crp_propagate(crp_context* c, const crp_grid* g, const crp_modules* m, void* stream,
                         crp_stats* stats_out) {
  if (!c || !g || !m) {
    set_error("crp_propagate: NULL argument");
    return CRP_E_INVALID;
  }
  if (g->ctx->device != c->device) {
    set_error("crp_propagate: grid belongs to another device");
    return CRP_E_INVALID;
  }
  if (m->precision != CRP_FP64 && m->precision != CRP_MIXED) {
    set_error("crp_propagate: precision must be CRP_FP64 or CRP_MIXED");
    return CRP_E_INVALID;
  }
  if (!(m->tol > 0.0) || !(m->h_min > 0.0) || !(m->h_max >= m->h_min) ||
      !(m->field_unit_T > 0.0) || !(m->length_unit_m > 0.0)) {
    set_error("crp_propagate: need tol > 0, 0 < h_min <= h_max, positive units");
    return CRP_E_INVALID;
  }
  const uint32_t need_tab = CRP_PAIR | CRP_PION | CRP_PHOTODIS;
  if ((m->flags & need_tab) && !m->tables) {
    set_error("crp_propagate: PAIR / PION / PHOTODIS need tables");
    return CRP_E_INVALID;
  }
  const int max_block = m->precision == CRP_FP64 ? 128 : 256;
  if (m->block_size < 0 || m->block_size > max_block || (m->block_size % 32) != 0 ||
      m->blocks_per_sm < 0) {
    set_error("crp_propagate: block_size must be a multiple of 32 up to %d", max_block);
    return CRP_E_INVALID;
  }
  if (m->queue_order < -1 || m->queue_order > 1) {
    set_error("crp_propagate: queue_order must be -1, 0 or 1");
    return CRP_E_INVALID;
  }
  if (m->precision == CRP_MIXED && !(m->h_max / g->desc.spacing < 1048576.0)) {
    set_error("crp_propagate: the mixed path needs a step to span fewer than 2^20 grid cells "
              "(h_max / spacing = %g)", m->h_max / g->desc.spacing);
    return CRP_E_INVALID;
  }
  if (stats_out) memset(stats_out, 0, sizeof(*stats_out));
  if (c->size == 0) return CRP_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  KParams kp;
  memset(&kp, 0, sizeof(kp));
  fill_field_view(g, kp.f);
  kp.tol = m->tol;
  kp.tol2 = m->tol * m->tol;
  kp.h_min = m->h_min;
  kp.h_max = m->h_max;
  kp.curv_k = 299792458.0 * m->field_unit_T * m->length_unit_m;
  kp.beta_ad = m->beta_ad;
  kp.e_min = m->e_min;
  kp.e_min_guard_f = (float)(m->e_min * 1.0001);
  // free-neutron decay length per eV (tau_n = 878.4 s, m_n c^2 = 939.56542052 MeV)
  kp.decay_k = 299792458.0 * 878.4 / 939.56542052e6 / m->length_unit_m;
  kp.length_unit_m = m->length_unit_m;
  kp.flags = m->flags;
  kp.seed = c->seed;
  if (m->tables && m->tables->nuc && (m->flags & CRP_DECAY)) {
    kp.nuc_tab = m->tables->nuc;
    kp.nuc_amax = m->tables->nuc_amax;
  }
  if (m->tables) {
    const crp_tables* t = m->tables;
    kp.t_beta = t->data;
    kp.t_pion = t->data + t->desc.n;
    kp.t_gdr = t->data + 2 * t->desc.n;
    kp.tab_lg0 = log(t->desc.gamma_lo);
    kp.tab_inv_dlg = (double)(t->desc.n - 1) / (log(t->desc.gamma_hi) - log(t->desc.gamma_lo));
    kp.tab_n = t->desc.n;
    kp.t_beta_f = t->data_f;
  } else {
    kp.tab_n = 2;
  }
  kp.tol2_f = (float)kp.tol2;
  kp.inv_tol2_f = (float)(1.0 / kp.tol2);
  kp.h_min_f = (float)kp.h_min;
  kp.h_max_f = (float)kp.h_max;
  kp.curv_k_f = (float)kp.curv_k;
  kp.beta_ad_f = (float)kp.beta_ad;
  kp.tab_lg0_f = (float)kp.tab_lg0;
  kp.tab_inv_dlg_f = (float)kp.tab_inv_dlg;
  fill_galactic(m, kp);
  if (crp_status gs = fill_gmf(m, kp, "crp_propagate")) return gs;
  for (int d = 0; d < 3; ++d) {
    kp.obs_c[d] = m->observer_center[d];
    kp.border_c[d] = m->border_center[d];
  }
  kp.obs_r = m->observer_radius;
  kp.border_r = m->border_radius;
  kp.max_steps = m->max_steps ? m->max_steps : 100000000ull;  // bound every candidate
  kp.step_budget = m->step_budget;
  kp.deadline_ns = m->deadline_ms > 0.0 ? (uint64_t)(m->deadline_ms * 1e6) : 0;
  kp.capacity = c->capacity;

  const int block = m->block_size ? m->block_size : (m->precision == CRP_FP64 ? 128 : 256);
  // mixed kernels come in three register budgets: 256 x 2 resident blocks
  // (128 registers), 128 x 5 (96) and 256 x 3 (80)
  int variant = 2;
  if (m->block_size && m->block_size <= 128)
    variant = (m->blocks_per_sm == 0 || m->blocks_per_sm <= 5) ? 5 : 3;
  else if (m->blocks_per_sm >= 3)
    variant = 3;
  // the analytic galactic fields' binary32 arithmetic is contracted
  // differently under the smaller register budgets, which would make the
  // records depend on the launch; those lists always run in the first
  if (m->flags & (CRP_GALACTIC | CRP_GMF)) variant = 2;
  int bps = m->blocks_per_sm;
  if (!bps) {
    cudaError_t e = m->precision == CRP_FP64
                        ? occupancy_propagate_fp64(kp.f.dtype, block, &bps, kp.nuc_tab != nullptr)
                        : occupancy_propagate_mixed(kp.f.dtype, m->flags,
                                                variant, block, &bps, kp.nuc_tab != nullptr);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: occupancy query");
    if (bps < 1) bps = 1;
  }

  if (c->size > 0xffffffffull) {
    set_error("crp_propagate: pool indices must fit 32 bits");
    return CRP_E_INVALID;
  }
  for (int d = 0; d < 3; ++d) {
    int bits = 0;
    while ((1ll << bits) < kp.f.n[d]) ++bits;
    kp.key_shift[d] = bits > 5 ? bits - 5 : 0;
  }
  kp.queue_order = m->queue_order;
  const bool sort_on = m->queue_order >= 0;
  const int3 shift3 = make_int3(kp.key_shift[0], kp.key_shift[1], kp.key_shift[2]);
  // Work queue of refill pass r is the list pass r-1 wrote (requeued candidates
  // and new secondaries), sorted by spatial brick; pass 0 lists the pool.
  uint32_t* q_in = c->queue[0];
  uint32_t* q_out = c->queue[1];
  auto sort_into_qin = [&](uint64_t n) -> cudaError_t {
    if (!sort_on || n < 8192) {
      std::swap(q_in, q_out);
      return cudaSuccess;
    }
    cudaError_t err = cudaMemsetAsync(c->bins, 0, (kSortBins + 1) * sizeof(uint32_t), s);
    if (err != cudaSuccess) return err;
    k_sort_hist<<<blocks_for(n, 256), 256, 0, s>>>(c->keys, n, c->bins);
    k_sort_scan<<<1, 1024, 0, s>>>(c->bins);
    k_sort_scatter<<<blocks_for(n, 256), 256, 0, s>>>(c->keys, q_out, n, c->bins, q_in);
    return cudaGetLastError();
  };
  cudaError_t e = cudaMemsetAsync(c->dc, 0, sizeof(DevCounters), s);
  if (e == cudaSuccess) {
    k_set_u64<<<1, 1, 0, s>>>(&c->dc->tail, (unsigned long long)c->size);
    k_build_queue<<<blocks_for(c->size, 256), 256, 0, s>>>(c->st, c->size, kp.f, shift3,
                                                           kp.queue_order, q_out, c->keys,
                                                           &c->dc->q_out);
    e = cudaGetLastError();
  }
  kp.slice = m->slice ? m->slice : kDefaultSlice;
  if (m->precision == CRP_MIXED && kp.slice % CRP_MIXED_REBASE_STEPS) {
    const uint64_t up = ((uint64_t)kp.slice / CRP_MIXED_REBASE_STEPS + 1) * CRP_MIXED_REBASE_STEPS;
    kp.slice = up > 0xffffffffull ? (0xffffffffu / CRP_MIXED_REBASE_STEPS) * CRP_MIXED_REBASE_STEPS
                                  : (uint32_t)up;
  }
  crp_status st = CRP_OK;
  uint32_t launches = 0;
  float total_ms = 0.f;
  if (m->use_graph) {
    // the queue the pre-loop built sits in queue[1]; the graph's first body
    // pass sorts it into queue[0] (fixed roles: no pointer swaps in a graph)
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: work queue");
    kp.queue_in = c->queue[0];
    kp.queue_out = c->queue[1];
    kp.keys_out = c->keys;
    kp.n_in = 0;
    kp.n_in_dev = &c->dc->n_in;
    e = graph_rounds(c, kp, m->precision, block, variant, c->sm_count * bps, sort_on, s,
                     &total_ms);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: graph");
    e = cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: graph counters");
    launches = (uint32_t)c->hc->rounds;
    if (c->hc->stop) {
      st = CRP_E_TIMEOUT;
      set_error("crp_propagate: step budget or deadline reached; candidates stay resumable");
    }
  }
  if (e == cudaSuccess && !m->use_graph)
    e = cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !m->use_graph) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: work queue");
  uint64_t n_in = m->use_graph ? 0 : c->hc->q_out;
  if (!m->use_graph) {
    e = sort_into_qin(n_in);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: queue sort");
  }
  while (n_in > 0) {
    kp.queue_in = q_in;
    kp.queue_out = q_out;
    kp.keys_out = c->keys;
    kp.n_in = n_in;
    uint64_t gsz = (uint64_t)c->sm_count * (uint64_t)bps;
    const uint64_t need = (n_in + block - 1) / block;
    if (need < gsz) gsz = need;
    k_round_reset<<<1, 1, 0, s>>>(c->dc);
    cudaEventRecord(c->ev0, s);
    e = m->precision == CRP_FP64 ? launch_propagate_fp64(kp, c->st, c->dc, (int)gsz, block, s)
                                 : launch_propagate_mixed(kp, c->st, c->dc, (int)gsz, block,
                                                          variant, s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: launch");
    cudaEventRecord(c->ev1, s);
    launches += 1;
    e = cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: kernel");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    total_ms += ms;
    if (c->hc->stop) {
      st = CRP_E_TIMEOUT;
      set_error("crp_propagate: step budget or deadline reached; candidates stay resumable");
      break;
    }
    n_in = c->hc->q_out < c->capacity ? c->hc->q_out : c->capacity;
    e = sort_into_qin(n_in);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate: queue sort");
  }
  uint64_t tail = c->hc->tail < c->capacity ? c->hc->tail : c->capacity;
  c->size = tail;
  if (st == CRP_OK && c->hc->overflow) {
    st = CRP_E_QUEUE_FULL;
    set_error("crp_propagate: %llu secondaries did not fit the pool capacity %zu",
              (unsigned long long)c->hc->overflow, c->capacity);
  }
  if (stats_out) {
    stats_out->accepted_steps = c->hc->acc;
    stats_out->rejected_trials = c->hc->rej;
    stats_out->rhs_evals = c->hc->rhs;
    stats_out->n_pion = c->hc->pion;
    stats_out->n_pd = c->hc->pd;
    stats_out->n_secondaries = c->hc->secondaries;
    stats_out->n_dropped = c->hc->dropped;
    stats_out->n_overflow = c->hc->overflow;
    stats_out->n_detected = c->hc->detected;
    stats_out->kernel_ms = total_ms;
    stats_out->launches = launches;
    stats_out->error_word = c->hc->error_word;
    // candidates still active (non-zero only after a timeout)
    if (st == CRP_E_TIMEOUT) {
      unsigned long long* cnt = &c->dc->head;
      cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
      k_count_active<<<blocks_for(c->size, 256), 256, 0, s>>>(c->st.status, c->size, cnt);
      cudaMemcpyAsync(&c->hc->head, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      stats_out->n_active = c->hc->head;
    }
  }
  return st;
}

// ---------------------------------------------------------------------------
crp_status crp_collect(crp_context* c, int32_t what, crp_record* out, size_t capacity,
                       size_t* n_out, int32_t out_on_device, void* stream) {
  if (!c || !n_out || (capacity && !out) || what < CRP_COLLECT_ALL || what > CRP_COLLECT_AT_BORDER) {
    set_error("crp_collect: bad argument");
    return CRP_E_INVALID;
  }
  *n_out = 0;
  if (c->size == 0) return CRP_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t n = c->size;
  const int nb = (int)((n + kCollectBlock - 1) / kCollectBlock);
  unsigned* counts = static_cast<unsigned*>(dev_alloc(sizeof(unsigned) * nb));
  unsigned long long* offs =
      static_cast<unsigned long long*>(dev_alloc(sizeof(unsigned long long) * (nb + 1)));
  crp_status st = CRP_OK;
  crp_record* tmp = nullptr;
  do {
    if (!counts || !offs) {
      st = CRP_E_OOM;
      set_error("crp_collect: allocation failed");
      break;
    }
    k_collect_count<<<nb, kCollectBlock, 0, s>>>(c->st.status, n, what, counts);
    k_collect_scan<<<1, 1024, 0, s>>>(counts, nb, offs);
    unsigned long long total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, offs + nb, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = fail_cuda(e, "crp_collect: count"); break; }
    *n_out = (size_t)total;
    if (total == 0 || (!out && capacity == 0)) break;  // size query
    if (total > capacity) {
      st = CRP_E_INVALID;
      set_error("crp_collect: %llu records selected, capacity %zu", total, capacity);
      break;
    }
    crp_record* dst = out;
    if (!out_on_device) {
      tmp = static_cast<crp_record*>(dev_alloc(sizeof(crp_record) * total));
      if (!tmp) { st = CRP_E_OOM; set_error("crp_collect: staging allocation failed"); break; }
      dst = tmp;
    }
    k_collect_scatter<<<nb, kCollectBlock, 0, s>>>(c->st, n, what, offs, dst);
    e = cudaGetLastError();
    if (e == cudaSuccess && !out_on_device)
      e = cudaMemcpyAsync(out, tmp, sizeof(crp_record) * total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = fail_cuda(e, "crp_collect"); break; }
  } while (0);
  dev_free(tmp);
  dev_free(counts);
  dev_free(offs);
  return st;
}

crp_status crp_histogram_energy(crp_context* c, int32_t what, double e_lo, double e_hi,
                                int32_t nbins, uint64_t* out, void* stream) {
  if (!c || !out || nbins < 1 || !(e_lo > 0.0) || !(e_hi > e_lo) || what < CRP_COLLECT_ALL ||
      what > CRP_COLLECT_AT_BORDER) {
    set_error("crp_histogram_energy: bad argument");
    return CRP_E_INVALID;
  }
  memset(out, 0, sizeof(uint64_t) * nbins);
  if (c->size == 0) return CRP_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* bins = static_cast<unsigned long long*>(dev_alloc(8 * (size_t)nbins));
  if (!bins) {
    set_error("crp_histogram_energy: allocation failed");
    return CRP_E_OOM;
  }
  const double l0 = log(e_lo), inv = (double)nbins / (log(e_hi) - l0);
  cudaError_t e = cudaMemsetAsync(bins, 0, 8 * (size_t)nbins, s);
  if (e == cudaSuccess) {
    k_hist_energy<<<blocks_for(c->size, 256), 256, 0, s>>>(c->st.status, c->st.E, c->size, what,
                                                           l0, inv, nbins, bins);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, bins, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(bins);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_histogram_energy");
}

crp_status crp_histogram_energy_device(crp_context* c, int32_t what, double e_lo, double e_hi,
                                       int32_t nbins, uint64_t* out_dev, int32_t accumulate,
                                       void* stream) {
  if (!c || !out_dev || nbins < 1 || !(e_lo > 0.0) || !(e_hi > e_lo) ||
      what < CRP_COLLECT_ALL || what > CRP_COLLECT_AT_BORDER) {
    set_error("crp_histogram_energy_device: bad argument");
    return CRP_E_INVALID;
  }
  DeviceGuard dg(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* bins = reinterpret_cast<unsigned long long*>(out_dev);
  cudaError_t e = cudaSuccess;
  if (!accumulate) e = cudaMemsetAsync(bins, 0, 8 * (size_t)nbins, s);
  if (e == cudaSuccess && c->size > 0) {
    const double l0 = log(e_lo), inv = (double)nbins / (log(e_hi) - l0);
    k_hist_energy<<<blocks_for(c->size, 256), 256, 0, s>>>(c->st.status, c->st.E, c->size, what,
                                                           l0, inv, nbins, bins);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "crp_histogram_energy_device");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// checkpoint / restore: the pool is the whole state of a propagation (every
// candidate carries its own RNG counters and free paths), so its first `size`
// entries of every array, with the seed, resume bit-identically.
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t n_arr;
  uint64_t seed;
  uint64_t size;
  uint64_t payload;
  uint64_t checksum;
  uint32_t elem[64];
};
constexpr char kCkptMagic[8] = {'C', 'R', 'P', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 2;

// FNV-1a over 32-bit words (every payload is a whole number of words).
uint64_t ckpt_hash(const unsigned char* p, size_t bytes) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t k = 0; k + 4 <= bytes; k += 4) {
    uint32_t w;
    memcpy(&w, p + k, 4);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

size_t ckpt_payload(const crp_context* c, uint64_t size) {
  size_t b = 0;
  for (int a = 0; a < c->n_arr; ++a) b += (size_t)c->arr_elem[a] * size;
  return b;
}

}  // namespace

extern "C" {

crp_status crp_checkpoint(crp_context* c, void* host_buf, size_t capacity, size_t* n_out,
                          void* stream) {
  if (!c || !n_out || (capacity && !host_buf)) {
    set_error("crp_checkpoint: bad argument");
    return CRP_E_INVALID;
  }
  DeviceGuard dg(c->device);
  crp_status st = ensure_pool(c);
  if (st != CRP_OK) return st;
  const size_t need = sizeof(CkptHeader) + ckpt_payload(c, c->size);
  *n_out = need;
  if (!host_buf) return CRP_OK;  // size query
  if (capacity < need) {
    set_error("crp_checkpoint: buffer holds %zu bytes, %zu needed", capacity, need);
    return CRP_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* out = static_cast<unsigned char*>(host_buf);
  unsigned char* p = out + sizeof(CkptHeader);
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < c->n_arr && e == cudaSuccess; ++a) {
    const size_t b = (size_t)c->arr_elem[a] * c->size;
    if (b) e = cudaMemcpyAsync(p, c->arr_ptr[a], b, cudaMemcpyDeviceToHost, s);
    p += b;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "crp_checkpoint");
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.version = kCkptVersion;
  h.n_arr = (uint32_t)c->n_arr;
  h.seed = c->seed;
  h.size = c->size;
  h.payload = need - sizeof(CkptHeader);
  for (int a = 0; a < c->n_arr; ++a) h.elem[a] = c->arr_elem[a];
  h.checksum = ckpt_hash(out + sizeof(CkptHeader), h.payload);
  memcpy(out, &h, sizeof(h));
  return CRP_OK;
}

crp_status crp_restore(crp_context* c, const void* host_buf, size_t n, void* stream) {
  if (!c || !host_buf || n < sizeof(CkptHeader)) {
    set_error("crp_restore: bad argument");
    return CRP_E_INVALID;
  }
  DeviceGuard dg(c->device);
  crp_status st = ensure_pool(c);
  if (st != CRP_OK) return st;
  CkptHeader h;
  memcpy(&h, host_buf, sizeof(h));
  const unsigned char* p = static_cast<const unsigned char*>(host_buf) + sizeof(CkptHeader);
  if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != kCkptVersion ||
      h.n_arr != (uint32_t)c->n_arr) {
    set_error("crp_restore: not a checkpoint of this library version");
    return CRP_E_INVALID;
  }
  for (int a = 0; a < c->n_arr; ++a) {
    if (h.elem[a] != c->arr_elem[a]) {
      set_error("crp_restore: array %d has element size %u, expected %u", a, h.elem[a],
                c->arr_elem[a]);
      return CRP_E_INVALID;
    }
  }
  if (h.size > c->capacity) {
    set_error("crp_restore: checkpoint holds %llu candidates, capacity is %zu",
              (unsigned long long)h.size, c->capacity);
    return CRP_E_INVALID;
  }
  if (h.payload != ckpt_payload(c, h.size) || n < sizeof(CkptHeader) + h.payload) {
    set_error("crp_restore: truncated checkpoint");
    return CRP_E_INVALID;
  }
  if (ckpt_hash(p, h.payload) != h.checksum) {
    set_error("crp_restore: checksum mismatch");
    return CRP_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < c->n_arr && e == cudaSuccess; ++a) {
    const size_t b = (size_t)c->arr_elem[a] * h.size;
    if (b) e = cudaMemcpyAsync(c->arr_ptr[a], p, b, cudaMemcpyHostToDevice, s);
    p += b;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "crp_restore");
  c->size = h.size;
  c->seed = h.seed;
  return CRP_OK;
}

}  // extern "C"

static_assert(sizeof(crp_record) == 208, "crp_record layout");
static_assert(sizeof(crp_stats) == 96, "crp_stats layout");

namespace crp {
void context_pool(const crp_context* c, DevState* st, uint64_t* n, int* device, uint64_t* seed) {
  *st = c->st;
  *n = c->pool ? c->size : 0;
  *device = c->device;
  *seed = c->seed;
}

// Work space of a context for other translation units: one index list of
// pool capacity (the first work queue, free outside crp_propagate) and a
// device counter.
void context_scratch(const crp_context* c, uint32_t** list, unsigned long long** counter) {
  *list = c->queue[0];
  *counter = c->dc ? &c->dc->lens_fallback : nullptr;
}

// Read-only view of a context's pool for other translation units of the
// library (status and energy arrays, pool size, device).
void context_view(const crp_context* c, const int32_t** status, const double** E, uint64_t* n,
                  int* device) {
  *status = c->st.status;
  *E = c->st.E;
  *n = c->pool ? c->size : 0;
  *device = c->device;
}
}  // namespace crp

// ---------------------------------------------------------------------------
// autotuner: time a few launch configurations on the context's own
// candidates (each from the same snapshot, each for a fixed number of
// accepted steps) and keep the fastest.  Results do not depend on the launch
// configuration (binary64 path: bit for bit; mixed path: slices are kept
// multiples of the mixed path's rebase period), so tuning changes only speed.
// ---------------------------------------------------------------------------
extern "C" crp_status crp_autotune(crp_context* c, const crp_grid* g, crp_modules* m,
                                   uint64_t steps_per_trial, crp_tune_result* out, void* stream) {
  if (!c || !g || !m || !out) {
    set_error("crp_autotune: NULL argument");
    return CRP_E_INVALID;
  }
  memset(out, 0, sizeof(*out));
  if (c->size == 0) {
    set_error("crp_autotune: inject the candidates to tune on first");
    return CRP_E_INVALID;
  }
  DeviceGuard dg(c->device);
  crp_status st = ensure_pool(c);
  if (st != CRP_OK) return st;
  // 0 or UINT64_MAX: score complete propagations (what a caller runs; a fixed
  // step budget sees only the steady state, not the end of the run)
  const bool whole_runs = steps_per_trial == 0 || steps_per_trial == ~0ull;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t size0 = c->size;
  const size_t bytes = ckpt_payload(c, size0);
  unsigned char* snap = static_cast<unsigned char*>(dev_alloc(bytes));
  if (!snap) {
    set_error("crp_autotune: cannot allocate the %zu-byte snapshot", bytes);
    return CRP_E_OOM;
  }
  auto copy_pool = [&](bool save) -> cudaError_t {
    size_t off = 0;
    for (int a = 0; a < c->n_arr; ++a) {
      const size_t b = (size_t)c->arr_elem[a] * size0;
      cudaError_t e = b ? cudaMemcpyAsync(save ? snap + off : c->arr_ptr[a],
                                          save ? c->arr_ptr[a] : snap + off, b,
                                          cudaMemcpyDeviceToDevice, s)
                        : cudaSuccess;
      if (e != cudaSuccess) return e;
      off += b;
    }
    c->size = size0;
    return cudaStreamSynchronize(s);
  };
  struct Cfg { int block, bps; uint32_t slice; int order; };
  Cfg cfgs[32];
  int nc = 0;
  const uint32_t slices[3] = {512u, 4096u, kDefaultSlice};
  const int mixed_bl[3][2] = {{256, 2}, {256, 3}, {128, 5}};
  const int fp64_bl[3][2] = {{128, 0}, {64, 0}, {32, 0}};
  for (int b = 0; b < 3; ++b) {
    const int* bl = m->precision == CRP_MIXED ? mixed_bl[b] : fp64_bl[b];
    for (uint32_t sl : slices)
      for (int order : {0, 1, -1}) cfgs[nc++] = Cfg{bl[0], bl[1], sl, order};
  }
  cudaError_t e = copy_pool(true);
  int best = -1;
  double best_rate = 0.0;
  for (int k = -1; k < nc && e == cudaSuccess && st == CRP_OK; ++k) {
    const Cfg& cf = cfgs[k < 0 ? 0 : k];  // k = -1: warm-up run, not scored
    crp_modules mm = *m;
    mm.block_size = cf.block;
    mm.blocks_per_sm = cf.bps;
    mm.slice = cf.slice;
    mm.queue_order = cf.order;
    mm.step_budget = whole_runs ? 0 : steps_per_trial;
    mm.deadline_ms = 0.0;
    crp_stats stt;
    const auto t0 = std::chrono::steady_clock::now();
    const crp_status r = crp_propagate(c, g, &mm, stream, &stt);
    const double dt =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (r != CRP_OK && r != CRP_E_TIMEOUT) {
      st = r;
      break;
    }
    e = copy_pool(false);
    if (k < 0) continue;
    const double rate = dt > 0.0 ? (double)stt.accepted_steps / dt : 0.0;
    if (rate > best_rate) {
      best_rate = rate;
      best = k;
    }
    out->n_tried += 1;
  }
  dev_free(snap);
  if (e != cudaSuccess) return fail_cuda(e, "crp_autotune");
  if (st != CRP_OK) return st;
  if (best >= 0) {
    m->block_size = cfgs[best].block;
    m->blocks_per_sm = cfgs[best].bps;
    m->slice = cfgs[best].slice;
    m->queue_order = cfgs[best].order;
    out->block_size = cfgs[best].block;
    out->blocks_per_sm = cfgs[best].bps;
    out->slice = cfgs[best].slice;
    out->queue_order = cfgs[best].order;
    out->steps_per_s = best_rate;
  }
  return CRP_OK;
}

// ---------------------------------------------------------------------------
// field sampling: the interpolated field exactly as the propagate kernels
// of the given precision evaluate it
// ---------------------------------------------------------------------------
extern "C" crp_status crp_grid_sample(const crp_grid* g, const crp_modules* m, int64_t n,
                                      const double* xyz, double* B_out) {
  if (!g || !m || n < 0 || (n && (!xyz || !B_out)) ||
      (m->precision != CRP_FP64 && m->precision != CRP_MIXED)) {
    set_error("crp_grid_sample: bad argument");
    return CRP_E_INVALID;
  }
  if (n == 0) return CRP_OK;
  DeviceGuard dg(g->ctx->device);
  KParams kp;
  memset(&kp, 0, sizeof(kp));
  fill_field_view(g, kp.f);
  kp.flags = m->flags & (CRP_GALACTIC | CRP_GMF);
  fill_galactic(m, kp);
  if (crp_status gs = fill_gmf(m, kp, "crp_grid_sample")) return gs;
  const size_t bytes = (size_t)n * 3 * sizeof(double);
  double* dx = static_cast<double*>(dev_alloc(bytes));
  double* dB = static_cast<double*>(dev_alloc(bytes));
  crp_status st = CRP_OK;
  if (!dx || !dB) {
    set_error("crp_grid_sample: device allocation failed");
    st = CRP_E_OOM;
  } else {
    cudaStream_t s = 0;
    cudaError_t e = cudaMemcpyAsync(dx, xyz, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = m->precision == CRP_FP64 ? sample_field_fp64(kp, dx, n, dB, s)
                                   : sample_field_mixed(kp, dx, n, dB, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B_out, dB, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail_cuda(e, "crp_grid_sample");
  }
  dev_free(dx);
  dev_free(dB);
  return st;
}

// ---------------------------------------------------------------------------
// 1D mode with cosmology and the a-posteriori correction
// ---------------------------------------------------------------------------
namespace {

struct Cosmo {
  double H0, omega_m, omega_l, dz_max, loss_max;  // H0 per length unit (H0 / c)
};

Cosmo cosmo_of(const crp_cosmology* c, double length_unit_m) {
  const double H0 = c && c->H0_km_s_Mpc > 0.0 ? c->H0_km_s_Mpc : 67.3;
  const double om = c && c->omega_m > 0.0 ? c->omega_m : 0.315;
  Cosmo k;
  k.H0 = H0 / 299792.458 * (length_unit_m / 3.0856775814913673e22);
  k.omega_m = om;
  k.omega_l = 1.0 - om;
  k.dz_max = c && c->dz_max > 0.0 ? c->dz_max : 1e-3;
  k.loss_max = c && c->loss_max > 0.0 ? c->loss_max : 1e-3;
  return k;
}

// Comoving distance to z: 16-point Gauss-Legendre on 64 panels of 1 / H.
double comoving_distance(const Cosmo& k, double z, const std::vector<double>& x,
                         const std::vector<double>& w) {
  const int panels = 64;
  const double width = z / panels;
  double total = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double mid = (p + 0.5) * width, half = 0.5 * width;
    double s = 0.0;
    for (size_t j = 0; j < x.size(); ++j) {
      const double a = 1.0 + mid + half * x[j];
      s += w[j] / (k.H0 * sqrt(k.omega_m * a * a * a + k.omega_l));
    }
    total += s * half;
  }
  return total;
}

// Redshift at comoving distance D: Newton's method on D(z) (dD/dz = 1/H)
// inside a bracket that every iterate narrows, bisection when Newton leaves it.
double redshift_at(const Cosmo& k, double D, const std::vector<double>& x,
                   const std::vector<double>& w) {
  if (D <= 0.0) return 0.0;
  double lo = 0.0, hi = 1.0;
  while (comoving_distance(k, hi, x, w) < D && hi < 1e6) hi *= 2.0;
  double z = D * k.H0;  // small-z start
  if (!(z > lo && z < hi)) z = 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double f = comoving_distance(k, z, x, w) - D;
    if (f < 0.0)
      lo = z;
    else
      hi = z;
    const double a = 1.0 + z;
    double zn = z - f * (k.H0 * sqrt(k.omega_m * a * a * a + k.omega_l));
    if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
    if (fabs(zn - z) <= 1e-16 * (1.0 + z) || hi - lo <= 1e-16 * hi) return zn;
    z = zn;
  }
  return z;
}

}  // namespace

extern "C" {

crp_status crp_redshift_of_distance(const crp_cosmology* cosmo, double length_unit_m, int64_t n,
                                    const double* D, double* z_out) {
  if (n < 0 || (n && (!D || !z_out)) || !(length_unit_m > 0.0)) {
    set_error("crp_redshift_of_distance: bad argument");
    return CRP_E_INVALID;
  }
  const Cosmo k = cosmo_of(cosmo, length_unit_m);
  std::vector<double> x, w;
  gauss_legendre(16, x, w);
  for (int64_t i = 0; i < n; ++i) {
    if (!(D[i] >= 0.0)) {
      set_error("crp_redshift_of_distance: distances must be >= 0");
      return CRP_E_INVALID;
    }
    z_out[i] = redshift_at(k, D[i], x, w);
  }
  return CRP_OK;
}

crp_status crp_propagate_1d(crp_context* c, const crp_cosmology* cosmo, const crp_modules* m,
                            void* stream, crp_stats* stats_out) {
  if (!c || !m) {
    set_error("crp_propagate_1d: NULL argument");
    return CRP_E_INVALID;
  }
  if ((m->flags & (CRP_PAIR | CRP_PION | CRP_PHOTODIS)) && !m->tables) {
    set_error("crp_propagate_1d: PAIR / PION / PHOTODIS need tables");
    return CRP_E_INVALID;
  }
  if (!(m->length_unit_m > 0.0)) {
    set_error("crp_propagate_1d: length_unit_m must be > 0");
    return CRP_E_INVALID;
  }
  if ((m->flags & CRP_DECAY) && m->tables && m->tables->nuc) {
    set_error("crp_propagate_1d: the 1D mode decays free neutrons only; use tables without a "
              "nuclide table (crp_tables_set_decay with n = 0)");
    return CRP_E_INVALID;
  }
  if (stats_out) memset(stats_out, 0, sizeof(*stats_out));
  if (c->size == 0) return CRP_OK;
  DeviceGuard dg(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Cosmo k = cosmo_of(cosmo, m->length_unit_m);
  K1dParams p;
  memset(&p, 0, sizeof(p));
  p.flags = m->flags;
  p.seed = c->seed;
  p.e_min = m->e_min;
  p.H0 = k.H0;
  p.omega_m = k.omega_m;
  p.omega_l = k.omega_l;
  p.dz_max = k.dz_max;
  p.loss_max = k.loss_max;
  if (m->tables) {
    const crp_tables* t = m->tables;
    p.t_beta = t->data;
    p.t_pion = t->data + t->desc.n;
    p.t_gdr = t->data + 2 * t->desc.n;
    p.tab_lg0 = log(t->desc.gamma_lo);
    p.tab_inv_dlg = (double)(t->desc.n - 1) / (log(t->desc.gamma_hi) - log(t->desc.gamma_lo));
    p.tab_n = t->desc.n;
  } else {
    p.tab_n = 2;
  }
  p.decay_k = 299792458.0 * 878.4 / 939.56542052e6 / m->length_unit_m;
  p.capacity = c->capacity;
  p.max_steps = m->max_steps ? m->max_steps : 100000000ull;
  const int block = 128;
  const int grid = c->sm_count * 8;
  uint32_t* q_in = c->queue[0];
  uint32_t* q_out = c->queue[1];
  const int3 shift3 = make_int3(0, 0, 0);
  FieldView none;
  memset(&none, 0, sizeof(none));
  none.n[0] = none.n[1] = none.n[2] = 1;
  cudaError_t e = cudaMemsetAsync(c->dc, 0, sizeof(DevCounters), s);
  if (e == cudaSuccess) {
    k_set_u64<<<1, 1, 0, s>>>(&c->dc->tail, (unsigned long long)c->size);
    k_build_queue<<<blocks_for(c->size, 256), 256, 0, s>>>(c->st, c->size, none, shift3, -1,
                                                           q_in, c->keys, &c->dc->q_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "crp_propagate_1d: work queue");
  uint64_t n_in = c->hc->q_out;
  uint32_t rounds = 0;
  float total_ms = 0.f;
  while (n_in > 0) {
    p.queue_in = q_in;
    p.queue_out = q_out;
    p.n_in = n_in;
    k_round_reset<<<1, 1, 0, s>>>(c->dc);
    cudaEventRecord(c->ev0, s);
    e = launch_propagate_1d(p, c->st, c->dc, grid, block, s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate_1d: launch");
    cudaEventRecord(c->ev1, s);
    rounds += 1;
    e = cudaMemcpyAsync(c->hc, c->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "crp_propagate_1d: kernel");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    total_ms += ms;
    n_in = c->hc->q_out < c->capacity ? c->hc->q_out : c->capacity;
    std::swap(q_in, q_out);
  }
  c->size = c->hc->tail < c->capacity ? c->hc->tail : c->capacity;
  crp_status st = CRP_OK;
  if (c->hc->overflow) {
    st = CRP_E_QUEUE_FULL;
    set_error("crp_propagate_1d: %llu secondaries did not fit the pool capacity %zu",
              (unsigned long long)c->hc->overflow, c->capacity);
  }
  if (stats_out) {
    stats_out->accepted_steps = c->hc->acc;
    stats_out->n_pion = c->hc->pion;
    stats_out->n_pd = c->hc->pd;
    stats_out->n_secondaries = c->hc->secondaries;
    stats_out->n_dropped = c->hc->dropped;
    stats_out->n_overflow = c->hc->overflow;
    stats_out->n_detected = c->hc->detected;
    stats_out->kernel_ms = total_ms;
    stats_out->launches = rounds;
    stats_out->error_word = c->hc->error_word;
  }
  return st;
}

crp_status crp_cosmology_pick(crp_context* ctx, const crp_cosmology* cosmo,
                              const crp_modules* m, int64_t n, const uint64_t* id,
                              const double* z_src, const double* E0, const int32_t* A0,
                              const int32_t* Z0, double* E_out, int32_t* A_out,
                              int32_t* Z_out, int32_t* n_products) {
  if (!ctx || !m || n < 0 ||
      (n && (!id || !z_src || !E0 || !A0 || !Z0 || !E_out || !A_out || !Z_out ||
             !n_products))) {
    set_error("crp_cosmology_pick: bad argument");
    return CRP_E_INVALID;
  }
  if (n == 0) return CRP_OK;
  for (int64_t i = 0; i < n; ++i) {
    if (!(z_src[i] >= 0.0) || !std::isfinite(z_src[i])) {
      set_error("crp_cosmology_pick: source redshift %lld is %g (must be finite and >= 0)",
                (long long)i, z_src[i]);
      return CRP_E_INVALID;
    }
  }
  std::vector<double> z(z_src, z_src + n);
  crp_status st = CRP_OK;
  int32_t amax = 1;
  for (int64_t i = 0; i < n; ++i) amax = A0[i] > amax ? A0[i] : amax;
  crp_context* c = nullptr;
  st = crp_context_create(ctx->device, ctx->seed, (size_t)n * (size_t)(amax + 1), &c);
  if (st != CRP_OK) return st;
  std::vector<double> zeros(n, 0.0), ones(n, 1.0);
  std::vector<int32_t> q(n, 1);
  crp_candidate_arrays a;
  memset(&a, 0, sizeof(a));
  a.id = id;
  a.x = z.data();
  a.y = zeros.data();
  a.z = zeros.data();
  a.ux = zeros.data();
  a.uy = zeros.data();
  a.uz = ones.data();
  a.E = E0;
  a.A = A0;
  a.Z = Z0;
  a.q = q.data();
  a.on_device = 0;
  st = crp_candidates_inject(c, &a, (size_t)n, 0, nullptr);
  if (st == CRP_OK) st = crp_propagate_1d(c, cosmo, m, nullptr, nullptr);
  std::vector<crp_record> rec;
  if (st == CRP_OK) {
    size_t cnt = 0;
    st = crp_collect(c, CRP_COLLECT_ALL, nullptr, 0, &cnt, 0, nullptr);
    if (st == CRP_OK) {
      rec.resize(cnt);
      st = crp_collect(c, CRP_COLLECT_ALL, rec.data(), cnt, &cnt, 0, nullptr);
      rec.resize(cnt);
    }
  }
  crp_context_destroy(c);
  if (st != CRP_OK) return st;
  // lineage root of every record: follow parent ids to a generation-0 record
  std::unordered_map<uint64_t, size_t> by_id;
  by_id.reserve(rec.size() * 2);
  for (size_t r = 0; r < rec.size(); ++r) by_id[rec[r].id] = r;
  std::unordered_map<uint64_t, std::vector<std::pair<uint64_t, size_t>>> products;
  for (size_t r = 0; r < rec.size(); ++r) {
    if (rec[r].status != CRP_DETECTED) continue;
    size_t cur = r;
    while (rec[cur].generation > 0) {
      auto it = by_id.find(rec[cur].parent_id);
      if (it == by_id.end()) break;
      cur = it->second;
    }
    products[rec[cur].id].push_back({rec[r].id, r});
  }
  for (int64_t i = 0; i < n; ++i) {
    auto it = products.find(id[i]);
    if (it == products.end() || it->second.empty()) {
      n_products[i] = 0;
      E_out[i] = 0.0;
      A_out[i] = 0;
      Z_out[i] = 0;
      continue;
    }
    auto& v = it->second;
    std::sort(v.begin(), v.end());
    const int64_t nk = (int64_t)v.size();
    const Philox4 w = draw4(ctx->seed, TAG_COSMOLOGY, id[i], 0);
    const double u = u01_open(w.v0, w.v1);
    int64_t k = (int64_t)floor(u * (double)nk);
    if (k > nk - 1) k = nk - 1;
    const crp_record& pick = rec[v[k].second];
    n_products[i] = (int32_t)nk;
    E_out[i] = pick.E;
    A_out[i] = pick.A;
    Z_out[i] = pick.Z;
  }
  return CRP_OK;
}

crp_status crp_cosmology_correct(crp_context* ctx, const crp_cosmology* cosmo,
                                 const crp_modules* m, int64_t n, const uint64_t* id,
                                 const double* T, const double* E0, const int32_t* A0,
                                 const int32_t* Z0, double* E_out, int32_t* A_out,
                                 int32_t* Z_out, int32_t* n_products) {
  if (!ctx || !m || n < 0 ||
      (n && (!id || !T || !E0 || !A0 || !Z0 || !E_out || !A_out || !Z_out || !n_products))) {
    set_error("crp_cosmology_correct: bad argument");
    return CRP_E_INVALID;
  }
  if (n == 0) return CRP_OK;
  std::vector<double> z(n);
  crp_status st = crp_redshift_of_distance(cosmo, m->length_unit_m, n, T, z.data());
  if (st != CRP_OK) return st;
  return crp_cosmology_pick(ctx, cosmo, m, n, id, z.data(), E0, A0, Z0, E_out, A_out, Z_out,
                            n_products);
}

}  // extern "C"
