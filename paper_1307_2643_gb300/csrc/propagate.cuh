// propagate.cuh -- the persistent propagate kernel.
//
// One thread owns one candidate at a time and runs the module list of
// CRPropa 3.0 (Sect. 3, Fig. 1) on it, one full cycle per loop iteration:
//   integration   Cash-Karp 5(4) trial steps of the Lorentz equation with
//                 trilinear field interpolation until the step controller
//                 accepts (Sect. 3: "deflects the particle ... updates the
//                 position, direction and trajectory length");
//   interactions  continuous pair-production and adiabatic losses; pion
//                 production and photodisintegration, each deciding
//                 independently, with all interaction states reset after any
//                 interaction and secondaries appended to the pool;
//   boundary / observer modules, then the IsActive check.
// Warps are persistent: when a lane's candidate stops, the warp hands the
// free lanes new pool slots with one atomic (ballot + popc), so candidates
// of very different path lengths share warps without idling them.
//
// Two precision policies:
//   FP64   every operation in binary64, in the same order as the reference
//          formulation of the method (compile this translation unit with
//          -fmad=false so no multiply-add is contracted);
//   MIXED  field interpolation, Lorentz force and RK stages in binary32;
//          position, trajectory length, energy, free paths and the error
//          norm in binary64.
#pragma once

#include <math.h>

#include "crp_internal.cuh"
#include "device_common.cuh"

namespace crp {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Node loads (float4 or DNode per grid node, x fastest).
// ---------------------------------------------------------------------------
template <class NodeT>
struct Node;

template <>
struct Node<float4> {
  __device__ __forceinline__ static void load(const void* base, size_t i, double& bx, double& by,
                                              double& bz) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(base) + i);
    bx = v.x;
    by = v.y;
    bz = v.z;
  }
  __device__ __forceinline__ static float4 loadf(const void* base, size_t i) {
    return __ldg(reinterpret_cast<const float4*>(base) + i);
  }
};

template <>
struct Node<DNode> {
  __device__ __forceinline__ static void load(const void* base, size_t i, double& bx, double& by,
                                              double& bz) {
    const double2* p = reinterpret_cast<const double2*>(base) + 2 * i;
    const double2 a = __ldg(p);
    const double2 b = __ldg(p + 1);
    bx = a.x;
    by = a.y;
    bz = b.x;
  }
  __device__ __forceinline__ static float4 loadf(const void* base, size_t i) {
    const double2* p = reinterpret_cast<const double2*>(base) + 2 * i;
    const double2 a = __ldg(p);
    const double2 b = __ldg(p + 1);
    return make_float4((float)a.x, (float)a.y, (float)b.x, 0.f);
  }
};

__device__ __forceinline__ int64_t wrap_fl(double fl, int64_t n, int64_t mask) {
  int64_t i = (int64_t)fl;
  if (mask >= 0) return i & mask;
  i = i % n;
  if (i < 0) i += n;
  return i;
}

__device__ __forceinline__ int wrap_int(int i, int n, int mask) {
  if (mask >= 0) return i & mask;
  i = i % n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ double lerp_d(double a, double b, double t) { return a + t * (b - a); }

// ---------------------------------------------------------------------------
// Analytic galactic field (disk log-spiral + toroidal halo), binary64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void galactic_fp64(const KParams& p, const double x[3], double G[3]) {
  const double rx = x[0] - p.gal_c[0], ry = x[1] - p.gal_c[1], z = x[2] - p.gal_c[2];
  const double r = sqrt(rx * rx + ry * ry);
  G[0] = 0.0;
  G[1] = 0.0;
  G[2] = 0.0;
  if (r == 0.0) return;
  const double cr = rx / r, sr = ry / r;
  const double az = fabs(z);
  double b_r = 0.0, b_phi = 0.0;
  if (r >= p.disk_rmin && r <= p.disk_rmax) {
    const double bd = p.disk_b * exp(-az / p.disk_hz);
    b_r += bd * p.sin_pitch;
    b_phi += bd * p.cos_pitch;
  }
  if (z != 0.0) {
    const double dz = az - p.halo_z0;
    const double bh = p.halo_b * exp(-dz * dz / (2.0 * p.halo_sigma * p.halo_sigma));
    b_phi += z > 0.0 ? bh : -bh;
  }
  G[0] = b_r * cr - b_phi * sr;
  G[1] = b_r * sr + b_phi * cr;
}

__device__ __forceinline__ float3 galactic_f32(const KParams& p, float rx, float ry, float z) {
  const float r2 = rx * rx + ry * ry;
  if (r2 == 0.f) return make_float3(0.f, 0.f, 0.f);
  const float ir = rsqrtf(r2);
  const float r = r2 * ir;
  const float cr = rx * ir, sr = ry * ir;
  const float az = fabsf(z);
  float b_r = 0.f, b_phi = 0.f;
  if (r >= (float)p.disk_rmin && r <= (float)p.disk_rmax) {
    const float bd = (float)p.disk_b * __expf(-az / (float)p.disk_hz);
    b_r = bd * (float)p.sin_pitch;
    b_phi = bd * (float)p.cos_pitch;
  }
  if (z != 0.f) {
    const float dz = az - (float)p.halo_z0;
    const float s = (float)p.halo_sigma;
    const float bh = (float)p.halo_b * __expf(-dz * dz / (2.f * s * s));
    b_phi += z > 0.f ? bh : -bh;
  }
  return make_float3(b_r * cr - b_phi * sr, b_r * sr + b_phi * cr, 0.f);
}

// ---------------------------------------------------------------------------
// FP64 field: trilinear on the periodic vertex-centred grid (nested lerps in
// x, then y, then z), plus the analytic galactic part when enabled.
// ---------------------------------------------------------------------------
template <class NodeT>
__device__ __forceinline__ void field_fp64(const KParams& p, const double x[3], double B[3]) {
  const FieldView& f = p.f;
  int64_t i0[3], i1[3];
  double t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double r = (x[d] - f.origin[d]) * f.inv_spacing;
    const double fl = floor(r);
    t[d] = r - fl;
    i0[d] = wrap_fl(fl, f.n[d], f.mask[d]);
    i1[d] = i0[d] + 1 == f.n[d] ? 0 : i0[d] + 1;
  }
  const size_t nx = (size_t)f.n[0], nxy = (size_t)f.n[0] * (size_t)f.n[1];
  const size_t zy00 = (size_t)i0[2] * nxy + (size_t)i0[1] * nx;
  const size_t zy01 = (size_t)i0[2] * nxy + (size_t)i1[1] * nx;
  const size_t zy10 = (size_t)i1[2] * nxy + (size_t)i0[1] * nx;
  const size_t zy11 = (size_t)i1[2] * nxy + (size_t)i1[1] * nx;
  double v[8][3];
  Node<NodeT>::load(f.data, zy00 + i0[0], v[0][0], v[0][1], v[0][2]);  // (x0, y0, z0)
  Node<NodeT>::load(f.data, zy00 + i1[0], v[1][0], v[1][1], v[1][2]);  // (x1, y0, z0)
  Node<NodeT>::load(f.data, zy01 + i0[0], v[2][0], v[2][1], v[2][2]);  // (x0, y1, z0)
  Node<NodeT>::load(f.data, zy01 + i1[0], v[3][0], v[3][1], v[3][2]);  // (x1, y1, z0)
  Node<NodeT>::load(f.data, zy10 + i0[0], v[4][0], v[4][1], v[4][2]);  // (x0, y0, z1)
  Node<NodeT>::load(f.data, zy10 + i1[0], v[5][0], v[5][1], v[5][2]);  // (x1, y0, z1)
  Node<NodeT>::load(f.data, zy11 + i0[0], v[6][0], v[6][1], v[6][2]);  // (x0, y1, z1)
  Node<NodeT>::load(f.data, zy11 + i1[0], v[7][0], v[7][1], v[7][2]);  // (x1, y1, z1)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double c00 = lerp_d(v[0][c], v[1][c], t[0]);
    const double c10 = lerp_d(v[2][c], v[3][c], t[0]);
    const double c01 = lerp_d(v[4][c], v[5][c], t[0]);
    const double c11 = lerp_d(v[6][c], v[7][c], t[0]);
    const double c0 = lerp_d(c00, c10, t[1]);
    const double c1 = lerp_d(c01, c11, t[1]);
    B[c] = lerp_d(c0, c1, t[2]);
  }
  if (p.flags & CRP_GALACTIC) {
    double G[3];
    galactic_fp64(p, x, G);
    B[0] = B[0] + G[0];
    B[1] = B[1] + G[1];
    B[2] = B[2] + G[2];
  }
}

template <class NodeT>
__device__ __forceinline__ void rhs_fp64(const KParams& p, const double y[6], double kappa,
                                         double k[6]) {
  double B[3];
  field_fp64<NodeT>(p, y, B);
  k[0] = y[3];
  k[1] = y[4];
  k[2] = y[5];
  const double cx = y[4] * B[2] - y[5] * B[1];
  const double cy = y[5] * B[0] - y[3] * B[2];
  const double cz = y[3] * B[1] - y[4] * B[0];
  k[3] = kappa * cx;
  k[4] = kappa * cy;
  k[5] = kappa * cz;
}

// ---------------------------------------------------------------------------
// Rate tables: linear interpolation in ln(Gamma), clamped.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double table_fp64(const KParams& p, const double* tab, double lng) {
  double t = (lng - p.tab_lg0) * p.tab_inv_dlg;
  const double tmax = (double)(p.tab_n - 1);
  if (t < 0.0) t = 0.0;
  if (t > tmax) t = tmax;
  int64_t i = (int64_t)floor(t);
  if (i > p.tab_n - 2) i = p.tab_n - 2;
  const double f = t - (double)i;
  const double a = __ldg(tab + i), b = __ldg(tab + i + 1);
  return a + f * (b - a);
}

__device__ __forceinline__ float table_f32(const KParams& p, const double* tab, float lng) {
  float t = (lng - (float)p.tab_lg0) * (float)p.tab_inv_dlg;
  const float tmax = (float)(p.tab_n - 1);
  t = fminf(fmaxf(t, 0.f), tmax);
  int i = (int)t;
  if (i > (int)p.tab_n - 2) i = (int)p.tab_n - 2;
  const float f = t - (float)i;
  const float a = (float)__ldg(tab + i), b = (float)__ldg(tab + i + 1);
  return fmaf(f, b - a, a);
}

// ---------------------------------------------------------------------------
// Per-lane candidate state and per-lane counters.
// ---------------------------------------------------------------------------
struct LaneCore {
  uint64_t id;
  uint64_t slot;
  double x[3];
  double E, s, s_max, h, d_pion, d_pd;
  int A, Z, q, status;
  uint32_t draws, events, n_pion, n_pd, n_dropped, flags;
  uint64_t n_acc, n_rej;
};

struct LaneFP64 : LaneCore {
  double u[3];
};

struct LaneMixed : LaneCore {
  float u[3];
  int cell[3];   // grid cell of the current position
  float frac[3]; // fractional position inside that cell (grid units)
  float gal[3];  // position relative to the galactic centre (binary32)
};

struct LaneCounters {
  uint64_t acc, rej, rhs, pion, pd, sec, dropped, detected;
  uint32_t pending_acc;
};

__device__ __forceinline__ void load_core(const DevState& st, uint64_t i, LaneCore& c) {
  c.slot = i;
  c.id = st.id[i];
  c.x[0] = st.x[i];
  c.x[1] = st.y[i];
  c.x[2] = st.z[i];
  c.E = st.E[i];
  c.s = st.s[i];
  c.s_max = st.s_max[i];
  c.h = st.h[i];
  c.d_pion = st.d_pion[i];
  c.d_pd = st.d_pd[i];
  c.A = st.A[i];
  c.Z = st.Z[i];
  c.q = st.q[i];
  c.status = st.status[i];
  c.draws = st.draws[i];
  c.events = st.events[i];
  c.n_pion = st.n_pion[i];
  c.n_pd = st.n_pd[i];
  c.n_dropped = st.n_dropped[i];
  c.flags = st.flags[i];
  c.n_acc = st.n_acc[i];
  c.n_rej = st.n_rej[i];
}

__device__ __forceinline__ void store_core(const DevState& st, const LaneCore& c) {
  const uint64_t i = c.slot;
  st.x[i] = c.x[0];
  st.y[i] = c.x[1];
  st.z[i] = c.x[2];
  st.E[i] = c.E;
  st.s[i] = c.s;
  st.h[i] = c.h;
  st.d_pion[i] = c.d_pion;
  st.d_pd[i] = c.d_pd;
  st.A[i] = c.A;
  st.Z[i] = c.Z;
  st.status[i] = c.status;
  st.draws[i] = c.draws;
  st.events[i] = c.events;
  st.n_pion[i] = c.n_pion;
  st.n_pd[i] = c.n_pd;
  st.n_dropped[i] = c.n_dropped;
  st.flags[i] = c.flags;
  st.n_acc[i] = c.n_acc;
  st.n_rej[i] = c.n_rej;
}

// ---------------------------------------------------------------------------
// Stochastic interactions (binary64 on both policies): draws, resets, events.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double draw_u(const KParams& p, LaneCore& c) {
  const Philox4 w = draw4(p.seed, TAG_INTERACTION, c.id, c.draws);
  c.draws += 1;
  return u01_open(w.v0, w.v1);
}

// Remaining free path d = -ln(u) / R(E) per interaction, in module order
// [pion production, photodisintegration], at the current energy.
__device__ __forceinline__ void reset_states(const KParams& p, LaneCore& c) {
  const double lng = log(c.E / ((double)c.A * MP_C2_EV));
  if (p.flags & CRP_PION) {
    const double u = draw_u(p, c);
    const double R = (double)c.A * table_fp64(p, p.t_pion, lng);
    c.d_pion = R > 0.0 ? -log(u) / R : (double)INFINITY;
  }
  if (p.flags & CRP_PHOTODIS) {
    const double u = draw_u(p, c);
    const double R = c.A >= 2 ? (double)c.A * table_fp64(p, p.t_gdr, lng) : 0.0;
    c.d_pd = R > 0.0 ? -log(u) / R : (double)INFINITY;
  }
  c.flags |= CF_STATES_DRAWN;
}

// Single-nucleon emission: proton with probability Z/A (kept away from
// Z' = 0 or N' = 0 daughters with A' >= 2); the nucleon carries E/A, the
// daughter E (A-1)/A; the nucleon is appended to the pool when E/A >= e_min.
template <class Lane>
__device__ __forceinline__ void photodisintegrate(const KParams& p, const DevState& st,
                                               DevCounters* dc, Lane& c, LaneCounters& lc,
                                               const double u_dir[3]) {
  const double u = draw_u(p, c);
  bool proton = u < (double)c.Z / (double)c.A;
  const int Ad = c.A - 1;
  if (proton && Ad >= 2 && c.Z - 1 == 0) proton = false;
  if (!proton && Ad >= 2 && Ad - c.Z == 0) proton = true;
  const double En = c.E / (double)c.A;
  const double Ed = c.E * (double)Ad / (double)c.A;
  if (!(p.flags & CRP_EMIN) || En >= p.e_min) {
    const unsigned long long slot = atomicAdd(&dc->tail, 1ull);
    if (slot < p.capacity) {
      const uint64_t cid = lineage_id(c.id, c.events);
      st.id[slot] = cid;
      st.parent[slot] = c.id;
      st.x[slot] = c.x[0];
      st.y[slot] = c.x[1];
      st.z[slot] = c.x[2];
      st.ux[slot] = u_dir[0];
      st.uy[slot] = u_dir[1];
      st.uz[slot] = u_dir[2];
      st.x0[slot] = c.x[0];
      st.y0[slot] = c.x[1];
      st.z0[slot] = c.x[2];
      st.ux0[slot] = u_dir[0];
      st.uy0[slot] = u_dir[1];
      st.uz0[slot] = u_dir[2];
      st.E[slot] = En;
      st.E0[slot] = En;
      st.s[slot] = c.s;
      st.s_max[slot] = c.s_max;
      st.h[slot] = p.h_max;
      st.d_pion[slot] = 0.0;
      st.d_pd[slot] = 0.0;
      st.A[slot] = 1;
      st.Z[slot] = proton ? 1 : 0;
      st.A0[slot] = 1;
      st.Z0[slot] = proton ? 1 : 0;
      st.q[slot] = c.q;
      st.status[slot] = CRP_ACTIVE;
      st.draws[slot] = 0;
      st.events[slot] = 0;
      st.generation[slot] = st.generation[c.slot] + 1;
      st.n_pion[slot] = 0;
      st.n_pd[slot] = 0;
      st.n_dropped[slot] = 0;
      st.flags[slot] = 0;
      st.lens_pixel[slot] = 0xffffffffu;
      st.n_acc[slot] = 0;
      st.n_rej[slot] = 0;
      lc.sec += 1;
    } else {
      atomicAdd(&dc->overflow, 1ull);
      atomicOr(&dc->error_word, ERR_QUEUE_FULL);
    }
  } else {
    c.n_dropped += 1;
    lc.dropped += 1;
  }
  c.A = Ad;
  c.Z = c.Z - (proton ? 1 : 0);
  c.E = Ed;
  c.n_pd += 1;
  c.events += 1;
  lc.pd += 1;
  reset_states(p, c);
}

// Does the segment a -> b enter the sphere (centre cen, radius R) from outside?
__device__ __forceinline__ bool segment_enters(const double a[3], const double b[3],
                                               const double cen[3], double R) {
  double f[3], d[3], g[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f[i] = a[i] - cen[i];
    d[i] = b[i] - a[i];
    g[i] = b[i] - cen[i];
  }
  const double R2 = R * R;
  const double fa = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
  if (fa <= R2) return false;
  const double gb = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  if (gb <= R2) return true;
  const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (dd == 0.0) return false;
  const double fd = f[0] * d[0] + f[1] * d[1] + f[2] * d[2];
  const double tstar = -fd / dd;
  if (!(tstar > 0.0 && tstar < 1.0)) return false;
  const double m2 = fa - fd * fd / dd;
  return m2 <= R2;
}

// Interaction modules + break conditions after an accepted step of length h.
// `x_old` is the position before the step; `u_dir` the direction after it.
template <class Lane, bool MIXED>
__device__ __forceinline__ void modules_after_step(const KParams& p, const DevState& st,
                                                   DevCounters* dc, Lane& c, LaneCounters& lc,
                                                   double h, const double x_old[3],
                                                   const double u_dir[3]) {
  const bool pion_on = (p.flags & CRP_PION) != 0;
  const bool pd_on = (p.flags & CRP_PHOTODIS) != 0;
  // continuous losses
  if (p.flags & (CRP_PAIR | CRP_ADIABATIC)) {
    if (MIXED) {
      float beta = 0.f;
      if (p.flags & CRP_PAIR) {
        const float g = (float)c.E / ((float)c.A * (float)MP_C2_EV);
        const float bp = table_f32(p, p.t_beta, __logf(g));
        beta = bp * (float)(c.Z * c.Z) / (float)c.A;
      }
      if (p.flags & CRP_ADIABATIC) beta += (float)p.beta_ad;
      c.E = c.E * (1.0 - (double)(beta * (float)h));
    } else {
      double beta = 0.0;
      if (p.flags & CRP_PAIR) {
        const double bp = table_fp64(p, p.t_beta, log(c.E / ((double)c.A * MP_C2_EV)));
        beta = bp * (double)(c.Z * c.Z) / (double)c.A;
      }
      if (p.flags & CRP_ADIABATIC) beta = beta + p.beta_ad;
      c.E = c.E * (1.0 - beta * h);
    }
  }
  // stochastic interactions
  if (pion_on || pd_on) {
    if (pion_on) c.d_pion = c.d_pion - h;
    if (pd_on) c.d_pd = c.d_pd - h;
    if (pion_on && c.d_pion <= 0.0) {
      c.E = c.E - 0.2 * c.E / (double)c.A;
      c.n_pion += 1;
      c.events += 1;
      lc.pion += 1;
      reset_states(p, c);
    } else if (pd_on && c.d_pd <= 0.0) {
      photodisintegrate(p, st, dc, c, lc, u_dir);
    }
  }
  // break conditions
  if ((p.flags & CRP_EMIN) && c.E < p.e_min) {
    c.status = CRP_BELOW_EMIN;
  } else if (c.s >= c.s_max) {
    c.status = CRP_MAX_LENGTH;
  } else if ((p.flags & CRP_OBSERVER) && segment_enters(x_old, c.x, p.obs_c, p.obs_r)) {
    c.status = CRP_DETECTED;
    lc.detected += 1;
  } else if (p.flags & CRP_BORDER) {
    const double dx = c.x[0] - p.border_c[0], dy = c.x[1] - p.border_c[1],
                 dz = c.x[2] - p.border_c[2];
    if (dx * dx + dy * dy + dz * dz >= p.border_r * p.border_r) c.status = CRP_AT_BORDER;
  }
  if (c.status == CRP_ACTIVE && p.max_steps && c.n_acc >= p.max_steps) c.status = CRP_BUDGET;
}

// ---------------------------------------------------------------------------
// FP64 policy: one module cycle.
// ---------------------------------------------------------------------------
struct PolicyFP64 {
  using Lane = LaneFP64;
  static constexpr bool kMixed = false;

  __device__ __forceinline__ static void load(const DevState& st, uint64_t i, Lane& c) {
    load_core(st, i, c);
    c.u[0] = st.ux[i];
    c.u[1] = st.uy[i];
    c.u[2] = st.uz[i];
  }
  __device__ __forceinline__ static void store(const DevState& st, const Lane& c) {
    store_core(st, c);
    st.ux[c.slot] = c.u[0];
    st.uy[c.slot] = c.u[1];
    st.uz[c.slot] = c.u[2];
  }

  template <class NodeT>
  __device__ __forceinline__ static void cycle(const KParams& p, const DevState& st,
                                               DevCounters* dc, Lane& c, LaneCounters& lc) {
    using namespace ck;
    const bool pion_on = (p.flags & CRP_PION) != 0;
    const bool pd_on = (p.flags & CRP_PHOTODIS) != 0;
    if ((pion_on || pd_on) && !(c.flags & CF_STATES_DRAWN)) reset_states(p, c);
    double h = c.h;
    if (h > p.h_max) h = p.h_max;
    const double cap_s = c.s_max - c.s;
    if (cap_s < h) h = cap_s;
    if (pion_on && c.d_pion < h) h = c.d_pion;
    if (pd_on && c.d_pd < h) h = c.d_pd;
    const double kappa = (double)(c.q * c.Z) * p.curv_k / c.E;
    const double y[6] = {c.x[0], c.x[1], c.x[2], c.u[0], c.u[1], c.u[2]};
    double k1[6], k2[6], k3[6], k4[6], k5[6], k6[6], yt[6], y5[6];
    rhs_fp64<NodeT>(p, y, kappa, k1);
    lc.rhs += 1;
    double eps;
    int rejections = 0;
    for (;;) {
#pragma unroll
      for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (a21 * k1[i]);
      rhs_fp64<NodeT>(p, yt, kappa, k2);
#pragma unroll
      for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (a31 * k1[i] + a32 * k2[i]);
      rhs_fp64<NodeT>(p, yt, kappa, k3);
#pragma unroll
      for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
      rhs_fp64<NodeT>(p, yt, kappa, k4);
#pragma unroll
      for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
      rhs_fp64<NodeT>(p, yt, kappa, k5);
#pragma unroll
      for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
      rhs_fp64<NodeT>(p, yt, kappa, k6);
      lc.rhs += 5;
#pragma unroll
      for (int i = 0; i < 6; ++i)
        y5[i] = y[i] + h * (w1 * k1[i] + w3 * k3[i] + w4 * k4[i] + w6 * k6[i]);
      double err[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        err[i] = h * (d1 * k1[3 + i] + d3 * k3[3 + i] + d4 * k4[3 + i] + d5 * k5[3 + i] +
                      d6 * k6[3 + i]);
      eps = sqrt(err[0] * err[0] + err[1] * err[1] + err[2] * err[2]) / p.tol;
      if (eps <= 1.0 || h <= p.h_min || rejections >= 64) break;
      double fac = 0.95 / sqrt(sqrt(eps));
      if (fac < 0.1) fac = 0.1;
      double hn = h * fac;
      if (hn < p.h_min) hn = p.h_min;
      h = hn;
      rejections += 1;
      c.n_rej += 1;
      lc.rej += 1;
    }
    const double x_old[3] = {c.x[0], c.x[1], c.x[2]};
    c.x[0] = y5[0];
    c.x[1] = y5[1];
    c.x[2] = y5[2];
    const double un = sqrt(y5[3] * y5[3] + y5[4] * y5[4] + y5[5] * y5[5]);
    const double inv = 1.0 / un;
    c.u[0] = y5[3] * inv;
    c.u[1] = y5[4] * inv;
    c.u[2] = y5[5] * inv;
    c.s = (h == cap_s) ? c.s_max : c.s + h;
    double grow = eps == 0.0 ? 5.0 : 0.95 / sqrt(sqrt(eps));
    if (grow > 5.0) grow = 5.0;
    double h_next = h * grow;
    if (h_next < p.h_min) h_next = p.h_min;
    if (h_next > p.h_max) h_next = p.h_max;
    c.h = h_next;
    c.n_acc += 1;
    lc.acc += 1;
    lc.pending_acc += 1;
    modules_after_step<Lane, false>(p, st, dc, c, lc, h, x_old, c.u);
  }
};

// ---------------------------------------------------------------------------
// Mixed policy: binary32 field / force / stages relative to the current cell.
// ---------------------------------------------------------------------------
struct PolicyMixed {
  using Lane = LaneMixed;
  static constexpr bool kMixed = true;

  // Cell index and in-cell fraction of the binary64 position; also the
  // binary32 offset from the galactic centre.
  __device__ __forceinline__ static void rebase(const KParams& p, Lane& c) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double r = (c.x[d] - p.f.origin[d]) * p.f.inv_spacing;
      const double fl = floor(r);
      c.frac[d] = (float)(r - fl);
      c.cell[d] = (int)wrap_fl(fl, p.f.n[d], p.f.mask[d]);
    }
    if (p.flags & CRP_GALACTIC) {
#pragma unroll
      for (int d = 0; d < 3; ++d) c.gal[d] = (float)(c.x[d] - p.gal_c[d]);
    }
  }

  __device__ __forceinline__ static void load(const DevState& st, uint64_t i, Lane& c,
                                              const KParams& p) {
    load_core(st, i, c);
    c.u[0] = (float)st.ux[i];
    c.u[1] = (float)st.uy[i];
    c.u[2] = (float)st.uz[i];
    rebase(p, c);
  }
  __device__ __forceinline__ static void store(const DevState& st, const Lane& c) {
    store_core(st, c);
    st.ux[c.slot] = (double)c.u[0];
    st.uy[c.slot] = (double)c.u[1];
    st.uz[c.slot] = (double)c.u[2];
  }

  // Field at the current position plus offset o (length unit).
  template <class NodeT>
  __device__ __forceinline__ static float3 field(const KParams& p, const Lane& c, float ox,
                                                 float oy, float oz) {
    const FieldView& f = p.f;
    const float rx = fmaf(ox, f.inv_spacing_f, c.frac[0]);
    const float ry = fmaf(oy, f.inv_spacing_f, c.frac[1]);
    const float rz = fmaf(oz, f.inv_spacing_f, c.frac[2]);
    const float fx = floorf(rx), fy = floorf(ry), fz = floorf(rz);
    const float tx = rx - fx, ty = ry - fy, tz = rz - fz;
    const int nx = (int)f.n[0], ny = (int)f.n[1], nz = (int)f.n[2];
    const int ix0 = wrap_int(c.cell[0] + (int)fx, nx, (int)f.mask[0]);
    const int iy0 = wrap_int(c.cell[1] + (int)fy, ny, (int)f.mask[1]);
    const int iz0 = wrap_int(c.cell[2] + (int)fz, nz, (int)f.mask[2]);
    const int ix1 = ix0 + 1 == nx ? 0 : ix0 + 1;
    const int iy1 = iy0 + 1 == ny ? 0 : iy0 + 1;
    const int iz1 = iz0 + 1 == nz ? 0 : iz0 + 1;
    const size_t snx = (size_t)nx, snxy = (size_t)nx * (size_t)ny;
    const size_t r00 = (size_t)iz0 * snxy + (size_t)iy0 * snx;
    const size_t r01 = (size_t)iz0 * snxy + (size_t)iy1 * snx;
    const size_t r10 = (size_t)iz1 * snxy + (size_t)iy0 * snx;
    const size_t r11 = (size_t)iz1 * snxy + (size_t)iy1 * snx;
    const float4 v0 = Node<NodeT>::loadf(f.data, r00 + ix0);
    const float4 v1 = Node<NodeT>::loadf(f.data, r00 + ix1);
    const float4 v2 = Node<NodeT>::loadf(f.data, r01 + ix0);
    const float4 v3 = Node<NodeT>::loadf(f.data, r01 + ix1);
    const float4 v4 = Node<NodeT>::loadf(f.data, r10 + ix0);
    const float4 v5 = Node<NodeT>::loadf(f.data, r10 + ix1);
    const float4 v6 = Node<NodeT>::loadf(f.data, r11 + ix0);
    const float4 v7 = Node<NodeT>::loadf(f.data, r11 + ix1);
    auto lerp = [](float a, float b, float t) { return fmaf(t, b - a, a); };
    float3 B;
    B.x = lerp(lerp(lerp(v0.x, v1.x, tx), lerp(v2.x, v3.x, tx), ty),
               lerp(lerp(v4.x, v5.x, tx), lerp(v6.x, v7.x, tx), ty), tz);
    B.y = lerp(lerp(lerp(v0.y, v1.y, tx), lerp(v2.y, v3.y, tx), ty),
               lerp(lerp(v4.y, v5.y, tx), lerp(v6.y, v7.y, tx), ty), tz);
    B.z = lerp(lerp(lerp(v0.z, v1.z, tx), lerp(v2.z, v3.z, tx), ty),
               lerp(lerp(v4.z, v5.z, tx), lerp(v6.z, v7.z, tx), ty), tz);
    if (p.flags & CRP_GALACTIC) {
      const float3 G = galactic_f32(p, c.gal[0] + ox, c.gal[1] + oy, c.gal[2] + oz);
      B.x += G.x;
      B.y += G.y;
      B.z += G.z;
    }
    return B;
  }

  __device__ __forceinline__ static float3 force(float kap, float ux, float uy, float uz,
                                                 float3 B) {
    return make_float3(kap * (uy * B.z - uz * B.y), kap * (uz * B.x - ux * B.z),
                       kap * (ux * B.y - uy * B.x));
  }

  template <class NodeT>
  __device__ __forceinline__ static void cycle(const KParams& p, const DevState& st,
                                               DevCounters* dc, Lane& c, LaneCounters& lc) {
    const bool pion_on = (p.flags & CRP_PION) != 0;
    const bool pd_on = (p.flags & CRP_PHOTODIS) != 0;
    if ((pion_on || pd_on) && !(c.flags & CF_STATES_DRAWN)) reset_states(p, c);
    double h = c.h;
    if (h > p.h_max) h = p.h_max;
    const double cap_s = c.s_max - c.s;
    if (cap_s < h) h = cap_s;
    if (pion_on && c.d_pion < h) h = c.d_pion;
    if (pd_on && c.d_pd < h) h = c.d_pd;
    const float kap = (float)(c.q * c.Z) * (float)p.curv_k / (float)c.E;
    constexpr float A21 = (float)ck::a21, A31 = (float)ck::a31, A32 = (float)ck::a32;
    constexpr float A41 = (float)ck::a41, A42 = (float)ck::a42, A43 = (float)ck::a43;
    constexpr float A51 = (float)ck::a51, A52 = (float)ck::a52, A53 = (float)ck::a53,
                    A54 = (float)ck::a54;
    constexpr float A61 = (float)ck::a61, A62 = (float)ck::a62, A63 = (float)ck::a63,
                    A64 = (float)ck::a64, A65 = (float)ck::a65;
    constexpr float W1 = (float)ck::w1, W3 = (float)ck::w3, W4 = (float)ck::w4,
                    W6 = (float)ck::w6;
    constexpr float D1 = (float)ck::d1, D3 = (float)ck::d3, D4 = (float)ck::d4,
                    D5 = (float)ck::d5, D6 = (float)ck::d6;
    const float u1x = c.u[0], u1y = c.u[1], u1z = c.u[2];
    const float3 k1 = force(kap, u1x, u1y, u1z, field<NodeT>(p, c, 0.f, 0.f, 0.f));
    lc.rhs += 1;
    float dxx, dxy, dxz, u5x, u5y, u5z;
    double err2;
    float e32 = 0.f;
    int rejections = 0;
    for (;;) {
      const float hf = (float)h;
      // stage 2
      const float u2x = fmaf(hf, A21 * k1.x, u1x), u2y = fmaf(hf, A21 * k1.y, u1y),
                  u2z = fmaf(hf, A21 * k1.z, u1z);
      const float3 k2 =
          force(kap, u2x, u2y, u2z, field<NodeT>(p, c, hf * A21 * u1x, hf * A21 * u1y, hf * A21 * u1z));
      // stage 3
      const float u3x = fmaf(hf, A31 * k1.x + A32 * k2.x, u1x),
                  u3y = fmaf(hf, A31 * k1.y + A32 * k2.y, u1y),
                  u3z = fmaf(hf, A31 * k1.z + A32 * k2.z, u1z);
      const float3 k3 = force(kap, u3x, u3y, u3z,
                              field<NodeT>(p, c, hf * (A31 * u1x + A32 * u2x),
                                           hf * (A31 * u1y + A32 * u2y),
                                           hf * (A31 * u1z + A32 * u2z)));
      // stage 4
      const float u4x = fmaf(hf, A41 * k1.x + A42 * k2.x + A43 * k3.x, u1x),
                  u4y = fmaf(hf, A41 * k1.y + A42 * k2.y + A43 * k3.y, u1y),
                  u4z = fmaf(hf, A41 * k1.z + A42 * k2.z + A43 * k3.z, u1z);
      const float3 k4 = force(kap, u4x, u4y, u4z,
                              field<NodeT>(p, c, hf * (A41 * u1x + A42 * u2x + A43 * u3x),
                                           hf * (A41 * u1y + A42 * u2y + A43 * u3y),
                                           hf * (A41 * u1z + A42 * u2z + A43 * u3z)));
      // stage 5
      const float u5sx = fmaf(hf, A51 * k1.x + A52 * k2.x + A53 * k3.x + A54 * k4.x, u1x),
                  u5sy = fmaf(hf, A51 * k1.y + A52 * k2.y + A53 * k3.y + A54 * k4.y, u1y),
                  u5sz = fmaf(hf, A51 * k1.z + A52 * k2.z + A53 * k3.z + A54 * k4.z, u1z);
      const float3 k5 = force(
          kap, u5sx, u5sy, u5sz,
          field<NodeT>(p, c, hf * (A51 * u1x + A52 * u2x + A53 * u3x + A54 * u4x),
                       hf * (A51 * u1y + A52 * u2y + A53 * u3y + A54 * u4y),
                       hf * (A51 * u1z + A52 * u2z + A53 * u3z + A54 * u4z)));
      // stage 6
      const float u6x = fmaf(hf, A61 * k1.x + A62 * k2.x + A63 * k3.x + A64 * k4.x + A65 * k5.x, u1x),
                  u6y = fmaf(hf, A61 * k1.y + A62 * k2.y + A63 * k3.y + A64 * k4.y + A65 * k5.y, u1y),
                  u6z = fmaf(hf, A61 * k1.z + A62 * k2.z + A63 * k3.z + A64 * k4.z + A65 * k5.z, u1z);
      const float3 k6 = force(
          kap, u6x, u6y, u6z,
          field<NodeT>(p, c, hf * (A61 * u1x + A62 * u2x + A63 * u3x + A64 * u4x + A65 * u5sx),
                       hf * (A61 * u1y + A62 * u2y + A63 * u3y + A64 * u4y + A65 * u5sy),
                       hf * (A61 * u1z + A62 * u2z + A63 * u3z + A64 * u4z + A65 * u5sz)));
      lc.rhs += 5;
      dxx = hf * (W1 * u1x + W3 * u3x + W4 * u4x + W6 * u6x);
      dxy = hf * (W1 * u1y + W3 * u3y + W4 * u4y + W6 * u6y);
      dxz = hf * (W1 * u1z + W3 * u3z + W4 * u4z + W6 * u6z);
      u5x = fmaf(hf, W1 * k1.x + W3 * k3.x + W4 * k4.x + W6 * k6.x, u1x);
      u5y = fmaf(hf, W1 * k1.y + W3 * k3.y + W4 * k4.y + W6 * k6.y, u1y);
      u5z = fmaf(hf, W1 * k1.z + W3 * k3.z + W4 * k4.z + W6 * k6.z, u1z);
      const float ex = hf * (D1 * k1.x + D3 * k3.x + D4 * k4.x + D5 * k5.x + D6 * k6.x);
      const float ey = hf * (D1 * k1.y + D3 * k3.y + D4 * k4.y + D5 * k5.y + D6 * k6.y);
      const float ez = hf * (D1 * k1.z + D3 * k3.z + D4 * k4.z + D5 * k5.z + D6 * k6.z);
      // error norm in binary64
      const double dex = ex, dey = ey, dez = ez;
      err2 = dex * dex + dey * dey + dez * dez;
      if (err2 <= p.tol2 || h <= p.h_min || rejections >= 64) break;
      e32 = (float)(err2 / p.tol2);
      float fac = 0.95f * rsqrtf(sqrtf(sqrtf(e32)));  // 0.95 eps^(-1/4)
      fac = fmaxf(fac, 0.1f);
      double hn = h * (double)fac;
      if (hn < p.h_min) hn = p.h_min;
      h = hn;
      rejections += 1;
      c.n_rej += 1;
      lc.rej += 1;
    }
    const double x_old[3] = {c.x[0], c.x[1], c.x[2]};
    c.x[0] = c.x[0] + (double)dxx;
    c.x[1] = c.x[1] + (double)dxy;
    c.x[2] = c.x[2] + (double)dxz;
    const float inv = rsqrtf(u5x * u5x + u5y * u5y + u5z * u5z);
    c.u[0] = u5x * inv;
    c.u[1] = u5y * inv;
    c.u[2] = u5z * inv;
    c.s = (h == cap_s) ? c.s_max : c.s + h;
    float grow = 5.f;
    if (err2 > 0.0) {
      e32 = (float)(err2 / p.tol2);
      grow = fminf(5.f, 0.95f * rsqrtf(sqrtf(sqrtf(e32))));
    }
    double h_next = h * (double)grow;
    if (h_next < p.h_min) h_next = p.h_min;
    if (h_next > p.h_max) h_next = p.h_max;
    c.h = h_next;
    c.n_acc += 1;
    lc.acc += 1;
    lc.pending_acc += 1;
    rebase(p, c);
    const double u_dir[3] = {(double)c.u[0], (double)c.u[1], (double)c.u[2]};
    modules_after_step<Lane, true>(p, st, dc, c, lc, h, x_old, u_dir);
  }
};

// ---------------------------------------------------------------------------
// Persistent driver.
// ---------------------------------------------------------------------------
template <class Policy>
__device__ __forceinline__ void policy_load(const DevState& st, uint64_t i,
                                            typename Policy::Lane& c, const KParams& p);
template <>
__device__ __forceinline__ void policy_load<PolicyFP64>(const DevState& st, uint64_t i,
                                                        LaneFP64& c, const KParams&) {
  PolicyFP64::load(st, i, c);
}
template <>
__device__ __forceinline__ void policy_load<PolicyMixed>(const DevState& st, uint64_t i,
                                                         LaneMixed& c, const KParams& p) {
  PolicyMixed::load(st, i, c, p);
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

template <class Policy, class NodeT>
__global__ void __launch_bounds__(256) propagate_kernel(const KParams p, const DevState st,
                                                        DevCounters* dc) {
  using Lane = typename Policy::Lane;
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = globaltimer_ns();
  Lane c;
  LaneCounters lc = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  bool has = false, exhausted = false;
  int iter = 0;
  for (;;) {
    // hand free lanes the next pool slots (one atomic per warp)
    const bool need = !has && !exhausted;
    const unsigned m = __ballot_sync(FULL_MASK, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&dc->head, (unsigned long long)__popc(m));
      base = __shfl_sync(FULL_MASK, base, leader);
      if (need) {
        const unsigned long long mine = base + __popc(m & ((1u << lane) - 1u));
        if (mine < p.hi) {
          if (st.status[mine] == CRP_ACTIVE) {
            policy_load<Policy>(st, mine, c, p);
            has = true;
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (__ballot_sync(FULL_MASK, has || !exhausted) == 0) break;
    if (has) {
      Policy::template cycle<NodeT>(p, st, dc, c, lc);
      if (c.status != CRP_ACTIVE) {
        Policy::store(st, c);
        has = false;
      }
    }
    if ((++iter & 31) == 0 && (p.step_budget || p.deadline_ns)) {
      const unsigned pend = __reduce_add_sync(FULL_MASK, lc.pending_acc);
      lc.pending_acc = 0;
      unsigned stop = 0;
      if (lane == 0) {
        const unsigned long long tot = atomicAdd(&dc->acc, (unsigned long long)pend) + pend;
        if (p.step_budget && tot >= p.step_budget) atomicExch(&dc->stop, 1u);
        if (p.deadline_ns && globaltimer_ns() - t0 > p.deadline_ns) atomicExch(&dc->stop, 1u);
        stop = *((volatile unsigned*)&dc->stop);
      }
      stop = __shfl_sync(FULL_MASK, stop, 0);
      if (stop) {
        if (has) Policy::store(st, c);  // still active: resumable
        break;
      }
    }
  }
  // fold lane counters into the call's totals
  const uint64_t acc_rem = warp_sum_u64((p.step_budget || p.deadline_ns) ? lc.pending_acc : lc.acc);
  const uint64_t rej = warp_sum_u64(lc.rej), rhs = warp_sum_u64(lc.rhs);
  const uint64_t pion = warp_sum_u64(lc.pion), pd = warp_sum_u64(lc.pd);
  const uint64_t sec = warp_sum_u64(lc.sec), dropped = warp_sum_u64(lc.dropped);
  const uint64_t det = warp_sum_u64(lc.detected);
  if (lane == 0) {
    if (acc_rem) atomicAdd(&dc->acc, (unsigned long long)acc_rem);
    if (rej) atomicAdd(&dc->rej, (unsigned long long)rej);
    atomicAdd(&dc->rhs, (unsigned long long)rhs);
    if (pion) atomicAdd(&dc->pion, (unsigned long long)pion);
    if (pd) atomicAdd(&dc->pd, (unsigned long long)pd);
    if (sec) atomicAdd(&dc->secondaries, (unsigned long long)sec);
    if (dropped) atomicAdd(&dc->dropped, (unsigned long long)dropped);
    if (det) atomicAdd(&dc->detected, (unsigned long long)det);
  }
}

template <class Policy>
cudaError_t launch_policy(const KParams& kp, const DevState& st, DevCounters* dc, int grid,
                          int block, cudaStream_t s) {
  if (kp.f.dtype == CRP_F32)
    propagate_kernel<Policy, float4><<<grid, block, 0, s>>>(kp, st, dc);
  else
    propagate_kernel<Policy, DNode><<<grid, block, 0, s>>>(kp, st, dc);
  return cudaGetLastError();
}

template <class Policy>
cudaError_t occupancy_policy(int dtype, int block, int* bps) {
  if (dtype == CRP_F32)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, propagate_kernel<Policy, float4>,
                                                         block, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, propagate_kernel<Policy, DNode>,
                                                       block, 0);
}

}  // namespace crp
