// propagate.cuh -- the persistent propagate kernel.
//
// One lane owns one candidate at a time and runs the module list of
// CRPropa 3.0 (Sect. 3, Fig. 1) on it:
//   integration   Cash-Karp 5(4) trial steps of the Lorentz equation with
//                 trilinear field interpolation until the step controller
//                 accepts (the integration module deflects the particle and
//                 updates position, direction and trajectory length);
//   interactions  continuous pair-production and adiabatic losses; pion
//                 production and photodisintegration, each deciding
//                 independently, with all interaction states reset after any
//                 interaction and secondaries appended to the pool;
//   boundary / observer modules, then the IsActive check.
// Scheduling (GB300 design, not from the paper): a warp advances one
// Cash-Karp trial per loop iteration for all its lanes, so the expensive
// stage loop runs converged; a lane keeps a candidate for at most `slice`
// accepted steps, then requeues it for the next round and takes the next
// queue entry (one atomic per warp: ballot + popc).  Candidates whose path
// lengths differ by orders of magnitude therefore share warps without
// idling them, and the imbalance at the end of a round is bounded by one
// slice.  Stage directions and forces live in shared memory (one column per
// thread), so the stage loop is not unrolled and the code stays small.
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

#include <type_traits>

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

// floor(r) for |r| < 2^22 without a conversion instruction: r + 1.5 * 2^23
// lies in [2^23, 2^24), where the binary32 spacing is 1, so the sum rounded
// toward -inf is 1.5 * 2^23 + floor(r) exactly; it gives floor(r) as a float
// (fl) and, from its bit pattern, as an integer.  Both equal floorf(r) and
// (int)floorf(r).  Outside that range the integer is meaningless but
// wrap_int still maps it into the grid.
__device__ __forceinline__ int floor_small(float r, float& fl) {
  constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
  const float s = __fadd_rd(r, kMagic);
  fl = s - kMagic;
  return __float_as_int(s) - 0x4B400000;  // bit pattern of 1.5 * 2^23
}

__device__ __forceinline__ int wrap_int(int i, int n, int mask) {
  if (mask >= 0) return i & mask;
  i = i % n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ double lerp_d(double a, double b, double t) { return a + t * (b - a); }

__device__ __forceinline__ uint32_t key_of_position(const KParams& p, double x, double y,
                                                    double z) {
  const double r[3] = {x, y, z};
  int c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    c[d] = (int)wrap_fl(floor((r[d] - p.f.origin[d]) * p.f.inv_spacing), p.f.n[d], p.f.mask[d]);
  return brick_key(c[0], c[1], c[2], p.key_shift);
}

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
    const double bd = p.disk_b * series_exp(-az / p.disk_hz);
    b_r += bd * p.sin_pitch;
    b_phi += bd * p.cos_pitch;
  }
  if (z != 0.0) {
    const double dz = az - p.halo_z0;
    const double bh = p.halo_b * series_exp(-dz * dz / (2.0 * p.halo_sigma * p.halo_sigma));
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
  if (r >= p.grmin && r <= p.grmax) {
    const float bd = p.gdisk_b * __expf(-az * p.ginv_hz);
    b_r = bd * p.gsin;
    b_phi = bd * p.gcos;
  }
  if (z != 0.f) {
    const float dz = az - p.ghalo_z0;
    const float bh = p.ghalo_b * __expf(-dz * dz * p.ghalo_inv2s2);
    b_phi += z > 0.f ? bh : -bh;
  }
  return make_float3(b_r * cr - b_phi * sr, b_r * sr + b_phi * cr, 0.f);
}

// ---------------------------------------------------------------------------
// Analytic multi-arm galactic field (CRP_GMF; the model is stated with
// crp_gmf in crp.h).  Binary64: every operation in the order of the model's
// statement, transcendentals by the series functions, so the field is
// reproducible bit for bit.  Binary32: fast intrinsics, for the mixed policy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double logistic_d(double t, double h, double w) {
  const double e = -2.0 * (fabs(t) - h) / w;
  if (e > 700.0) return 0.0;
  return 1.0 / (1.0 + series_exp(e));
}

// Arm holding the logarithmic spiral through (r, phi): the spiral's crossing
// of phi = pi, ln r_x = ln r + (pi - phi) tan p, reduced modulo 2 pi tan p
// above ln arm_rx[0], and the last arm boundary at or below it.
template <class T>
__device__ __forceinline__ T arm_strength(const T (&arm_b)[8], const T (&d_arm)[8], T t) {
  T b = arm_b[0];
#pragma unroll
  for (int j = 1; j < 8; ++j)
    if (t >= d_arm[j]) b = arm_b[j];
  return b;
}

__device__ __forceinline__ void gmf_fp64(const KParams& p, const double x[3], double G[3]) {
  const GmfView& g = p.gm;
  const double rx = x[0] - p.gal_c[0], ry = x[1] - p.gal_c[1], z = x[2] - p.gal_c[2];
  G[0] = 0.0;
  G[1] = 0.0;
  G[2] = 0.0;
  const double R2 = rx * rx + ry * ry + z * z;
  if (g.cut_in2 > 0.0 && R2 < g.cut_in2) return;
  if (g.cut_out2 > 0.0 && R2 > g.cut_out2) return;
  const double r = sqrt(rx * rx + ry * ry);
  const double az = fabs(z);
  const double l_disk = logistic_d(z, g.h_disk, g.w_disk);
  double b_r = 0.0, b_phi = 0.0, b_z = 0.0;
  if (r >= g.r_ring && r <= g.r_out && r > 0.0) {
    if (r < g.r_in) {
      b_phi += g.ring_b * (1.0 - l_disk);
    } else {
      const double pi = 3.14159265358979323846;
      const double phi = series_atan2(ry, rx);
      double t = series_log(r) + (pi - phi) * g.tan_p - g.ln_r0;
      t = t - floor(t / g.period) * g.period;
      if (t < 0.0) t = t + g.period;
      if (t >= g.period) t = t - g.period;
      const double bd = arm_strength(g.arm_b, g.d_arm, t) * (g.r_in / r) * (1.0 - l_disk);
      b_r += bd * g.sin_p;
      b_phi += bd * g.cos_p;
    }
  }
  const double bh = z >= 0.0 ? g.halo_bn * (1.0 - logistic_d(r, g.halo_rn, g.halo_wh))
                             : g.halo_bs * (1.0 - logistic_d(r, g.halo_rs, g.halo_wh));
  b_phi += series_exp(-az / g.halo_z0) * l_disk * bh;
  if (g.x_b != 0.0) {
    const double rp_out = r - az / g.tan_t;
    double bx, sin_e, cos_e;
    if (rp_out >= g.x_rc) {
      bx = g.x_b * series_exp(-rp_out / g.x_r) * (rp_out / r);
      sin_e = g.sin_t;
      cos_e = g.cos_t;
    } else {
      const double f = g.x_rc / (g.x_rc + az / g.tan_t);
      const double rp = r * f;
      bx = g.x_b * series_exp(-rp / g.x_r) * (f * f);
      const double q = g.x_rc * g.tan_t;  // tan(elevation) = q / r_p
      const double nrm = sqrt(rp * rp + q * q);
      sin_e = q / nrm;
      cos_e = rp / nrm;
    }
    b_z += bx * sin_e;
    if (z > 0.0) b_r += bx * cos_e;
    if (z < 0.0) b_r -= bx * cos_e;
  }
  if (r > 0.0) {
    const double cr = rx / r, sr = ry / r;
    G[0] = b_r * cr - b_phi * sr;
    G[1] = b_r * sr + b_phi * cr;
  }
  G[2] = b_z;
}

__device__ __forceinline__ float3 gmf_f32(const KParams& p, float rx, float ry, float z) {
  const GmfView& g = p.gm;
  const float rr2 = rx * rx + ry * ry;
  const float R2 = rr2 + z * z;
  if (R2 < g.f_cut_in2 || (g.f_cut_out2 > 0.f && R2 > g.f_cut_out2))
    return make_float3(0.f, 0.f, 0.f);
  const float az = fabsf(z);
  // 1 / (1 + e^{-2 (|t| - h) / w}); an overflowing exponential gives 0
  const float l_disk = 1.f / (1.f + __expf((az - g.f_h_disk) * g.f_m2_inv_w_disk));
  float b_r = 0.f, b_phi = 0.f, b_z = 0.f;
  const float ir = rr2 > 0.f ? rsqrtf(rr2) : 0.f;
  const float r = rr2 * ir;
  if (r >= g.f_r_ring && r <= g.f_r_out && r > 0.f) {
    if (r < g.f_r_in) {
      b_phi = g.f_ring_b * (1.f - l_disk);
    } else {
      const float phi = atan2f(ry, rx);
      float t = __logf(r) + (3.14159265f - phi) * g.f_tan_p - g.f_ln_r0;
      t -= floorf(t * g.f_inv_period) * g.f_period;
      if (t < 0.f) t += g.f_period;
      if (t >= g.f_period) t -= g.f_period;
      const float bd = arm_strength(g.f_arm_b, g.f_d_arm, t) * (g.f_r_in * ir) * (1.f - l_disk);
      b_r = bd * g.f_sin_p;
      b_phi = bd * g.f_cos_p;
    }
  }
  const bool north = z >= 0.f;
  const float b0 = north ? g.f_halo_bn : g.f_halo_bs;
  const float rh = north ? g.f_halo_rn : g.f_halo_rs;
  const float bh = b0 * (1.f - 1.f / (1.f + __expf((r - rh) * g.f_m2_inv_halo_wh)));
  b_phi += __expf(-az * g.f_inv_halo_z0) * l_disk * bh;
  if (g.f_x_b != 0.f) {
    const float rp_out = r - az * g.f_inv_tan_t;
    float bx, sin_e, cos_e;
    if (rp_out >= g.f_x_rc) {
      bx = g.f_x_b * __expf(-rp_out * g.f_inv_x_r) * (rp_out * ir);
      sin_e = g.f_sin_t;
      cos_e = g.f_cos_t;
    } else {
      const float f = __fdividef(g.f_x_rc, g.f_x_rc + az * g.f_inv_tan_t);
      const float rp = r * f;
      bx = g.f_x_b * __expf(-rp * g.f_inv_x_r) * (f * f);
      const float inrm = rsqrtf(rp * rp + g.f_q * g.f_q);
      sin_e = g.f_q * inrm;
      cos_e = rp * inrm;
    }
    b_z = bx * sin_e;
    b_r += z > 0.f ? bx * cos_e : (z < 0.f ? -bx * cos_e : 0.f);
  }
  const float cr = rx * ir, sr = ry * ir;
  return make_float3(b_r * cr - b_phi * sr, b_r * sr + b_phi * cr, b_z);
}

// Dynamic shared memory of the propagate kernels (FP64: stage vectors;
// mixed: per-lane cell-record cache).
extern __shared__ __align__(16) unsigned char crp_dyn_smem[];

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
  if (p.flags & CRP_GMF) {
    double G[3];
    gmf_fp64(p, x, G);
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

__device__ __forceinline__ float table_f32(const KParams& p, const float* tab, float lng) {
  float t = (lng - p.tab_lg0_f) * p.tab_inv_dlg_f;
  const float tmax = (float)(p.tab_n - 1);
  t = fminf(fmaxf(t, 0.f), tmax);
  int i = (int)t;
  if (i > (int)p.tab_n - 2) i = (int)p.tab_n - 2;
  const float f = t - (float)i;
  const float a = __ldg(tab + i), b = __ldg(tab + i + 1);
  return fmaf(f, b - a, a);
}

// ---------------------------------------------------------------------------
// Candidate state as the rare paths (interaction draws, pion production,
// photodisintegration) see it.  These run on the candidate's slot in global
// memory, out of line, so the hot lane state below stays in registers.
// ---------------------------------------------------------------------------
struct EvCore {
  uint64_t id, slot;
  double x[3];
  double E, s, s_max, d_pion, d_pd, d_dec;
  int A, Z, q;
  uint32_t draws, events, n_pion, n_pd, n_dropped, flags;
};

struct EvCounts {
  uint32_t pion, pd, sec, dropped;
};

__device__ __forceinline__ double draw_u(const KParams& p, EvCore& c) {
  const Philox4 w = draw4(p.seed, TAG_INTERACTION, c.id, c.draws);
  c.draws += 1;
  return u01_open(w.v0, w.v1);
}

// Table entry of an unstable nucleus (A >= 2): [tau (s), cumulative branching
// after beta-, after beta+, after neutron emission, channel past the last
// sum], or null (stable, or no table).
__device__ __forceinline__ const double* nuclide(const KParams& p, int A, int Z) {
  if (!p.nuc_tab || A < 2 || A > p.nuc_amax || Z < 0 || Z > A) return nullptr;
  return p.nuc_tab + kNucEntry * ((int64_t)A * (A + 1) / 2 + Z);
}

// Remaining free path d = -ln(u) / R(E) per interaction, in module order
// [pion production, photodisintegration, decay], at the current energy.
// NUC: kernels launched with a nuclide table; the others never see one, and
// their rare paths are compiled without it.
template <bool NUC>
__device__ __forceinline__ void reset_states(const KParams& p, EvCore& c) {
  const double lng = series_log(c.E / ((double)c.A * MP_C2_EV));
  if (p.flags & CRP_PION) {
    const double u = draw_u(p, c);
    const double R = (double)c.A * table_fp64(p, p.t_pion, lng);
    c.d_pion = R > 0.0 ? -series_log(u) / R : (double)INFINITY;
  }
  if (p.flags & CRP_PHOTODIS) {
    const double u = draw_u(p, c);
    const double R = c.A >= 2 ? (double)c.A * table_fp64(p, p.t_gdr, lng) : 0.0;
    c.d_pd = R > 0.0 ? -series_log(u) / R : (double)INFINITY;
  }
  if (p.flags & CRP_DECAY) {
    // free neutrons decay after -ln(u) gamma c tau; drawn for every species.
    // With a nuclide table, an unstable nucleus after -ln(u) gamma c tau with
    // gamma = E / (A m_p c^2).
    const double u = draw_u(p, c);
    if (c.A == 1 && c.Z == 0) {
      c.d_dec = -series_log(u) * (c.E * p.decay_k);
    } else if (!NUC) {
      c.d_dec = (double)INFINITY;
    } else {
      const double* e = nuclide(p, c.A, c.Z);
      c.d_dec = (e && e[0] < (double)INFINITY)
                    ? -series_log(u) *
                          (c.E * (299792458.0 * e[0] / ((double)c.A * MP_C2_EV) / p.length_unit_m))
                    : (double)INFINITY;
    }
  }
  c.flags |= CF_STATES_DRAWN;
}

// Neutron beta decay: n -> p e nu; the proton keeps the Lorentz factor.
template <bool NUC>
__device__ __forceinline__ void decay_event(const KParams& p, EvCore& c) {
  c.Z = 1;
  c.E = c.E * (MP_C2_EV / MN_C2_EV);
  c.events += 1;
  reset_states<NUC>(p, c);
}

// Pion event: one nucleon loses the inelasticity 0.2 of its energy.
template <bool NUC>
__device__ __forceinline__ void pion_event(const KParams& p, EvCore& c, EvCounts& n) {
  c.E = c.E - 0.2 * c.E / (double)c.A;
  c.n_pion += 1;
  c.events += 1;
  n.pion += 1;
  reset_states<NUC>(p, c);
}

// Single-nucleon emission: proton with probability Z/A (kept away from
// Z' = 0 or N' = 0 daughters with A' >= 2); the nucleon carries E/A, the
// daughter E (A-1)/A; the nucleon is appended to the pool, and to the next
// round's work queue, when E/A >= e_min.
// Append an emitted nucleon of energy En at the candidate's position,
// direction and trajectory length (lineage id from the candidate's event
// count), and queue it for the next round; below e_min it is only counted.
__device__ __forceinline__ void emit_nucleon(const KParams& p, const DevState& st,
                                             DevCounters* dc, EvCore& c, EvCounts& n,
                                             bool proton, double En, double ux, double uy,
                                             double uz) {
  if (!(p.flags & CRP_EMIN) || En >= p.e_min) {
    const unsigned long long slot = atomicAdd(&dc->tail, 1ull);
    if (slot < p.capacity) {
      st.id[slot] = lineage_id(c.id, c.events);
      st.parent[slot] = c.id;
      st.x[slot] = c.x[0];
      st.y[slot] = c.x[1];
      st.z[slot] = c.x[2];
      st.ux[slot] = ux;
      st.uy[slot] = uy;
      st.uz[slot] = uz;
      st.x0[slot] = c.x[0];
      st.y0[slot] = c.x[1];
      st.z0[slot] = c.x[2];
      st.ux0[slot] = ux;
      st.uy0[slot] = uy;
      st.uz0[slot] = uz;
      st.E[slot] = En;
      st.E0[slot] = En;
      st.s[slot] = c.s;
      st.s_max[slot] = c.s_max;
      st.h[slot] = p.h_max;
      st.d_pion[slot] = 0.0;
      st.d_pd[slot] = 0.0;
      st.d_dec[slot] = 0.0;
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
      // the nucleon joins the next round (its slot is fully written first)
      const unsigned long long qo = atomicAdd(&dc->q_out, 1ull);
      if (qo < p.capacity) {
        p.queue_out[qo] = (uint32_t)slot;
        p.keys_out[qo] = p.queue_order == 1 ? key_of_position(p, c.x[0], c.x[1], c.x[2])
                                             : rigidity_key(En, proton ? 1 : 0);
      }
      n.sec += 1;
    } else {
      atomicAdd(&dc->overflow, 1ull);
      atomicOr(&dc->error_word, ERR_QUEUE_FULL);
    }
  } else {
    c.n_dropped += 1;
    n.dropped += 1;
  }
}

template <bool NUC>
__device__ __forceinline__ void photodisintegrate(const KParams& p, const DevState& st,
                                                  DevCounters* dc, EvCore& c, EvCounts& n,
                                                  double ux, double uy, double uz) {
  const double u = draw_u(p, c);
  bool proton = u < (double)c.Z / (double)c.A;
  const int Ad = c.A - 1;
  if (proton && Ad >= 2 && c.Z - 1 == 0) proton = false;
  if (!proton && Ad >= 2 && Ad - c.Z == 0) proton = true;
  const double En = c.E / (double)c.A;
  const double Ed = c.E * (double)Ad / (double)c.A;
  emit_nucleon(p, st, dc, c, n, proton, En, ux, uy, uz);
  c.A = Ad;
  c.Z = c.Z - (proton ? 1 : 0);
  c.E = Ed;
  c.n_pd += 1;
  c.events += 1;
  n.pd += 1;
  reset_states<NUC>(p, c);
}

// Decay of an unstable nucleus: one uniform picks the channel by the
// cumulative branching fractions (beta-, beta+, neutron emission, proton
// emission).  beta-+ change Z by +-1 and keep the energy (mass A m_p; the
// leptons are not followed); nucleon emission splits the energy as
// photodisintegration does (nucleon E / A, daughter E (A - 1) / A).
template <bool NUC>
__device__ __forceinline__ void nuclear_decay(const KParams& p, const DevState& st,
                                              DevCounters* dc, EvCore& c, EvCounts& n,
                                              double ux, double uy, double uz) {
  const double* e = nuclide(p, c.A, c.Z);
  const double u = draw_u(p, c);
  const int ch = u < e[1] ? 0 : (u < e[2] ? 1 : (u < e[3] ? 2 : (int)e[4]));
  if (ch == 0) {
    c.Z = c.Z + 1;
  } else if (ch == 1) {
    c.Z = c.Z - 1;
  } else {
    const bool proton = ch == 3;
    const int Ad = c.A - 1;
    const double En = c.E / (double)c.A;
    const double Ed = c.E * (double)Ad / (double)c.A;
    emit_nucleon(p, st, dc, c, n, proton, En, ux, uy, uz);
    c.A = Ad;
    c.Z = c.Z - (proton ? 1 : 0);
    c.E = Ed;
  }
  c.events += 1;
  reset_states<NUC>(p, c);
}

enum : int { EV_NONE = 0, EV_PION = 1, EV_PD = 2, EV_DRAW = 3, EV_DECAY = 4 };

// Run one rare path on the slot: first free-path draw (EV_DRAW), a pion
// event, a photodisintegration event or a decay.
template <bool NUC>
static __device__ __noinline__ void slot_event(const KParams& p, const DevState& st, DevCounters* dc,
                                        uint64_t i, int kind) {
  EvCore c;
  c.slot = i;
  c.id = st.id[i];
  c.x[0] = st.x[i];
  c.x[1] = st.y[i];
  c.x[2] = st.z[i];
  c.E = st.E[i];
  c.s = st.s[i];
  c.s_max = st.s_max[i];
  c.d_pion = st.d_pion[i];
  c.d_pd = st.d_pd[i];
  c.d_dec = st.d_dec[i];
  c.A = st.A[i];
  c.Z = st.Z[i];
  c.q = st.q[i];
  c.draws = st.draws[i];
  c.events = st.events[i];
  c.n_pion = st.n_pion[i];
  c.n_pd = st.n_pd[i];
  c.n_dropped = st.n_dropped[i];
  c.flags = st.flags[i];
  EvCounts n = {0, 0, 0, 0};
  if (kind == EV_PION)
    pion_event<NUC>(p, c, n);
  else if (kind == EV_PD)
    photodisintegrate<NUC>(p, st, dc, c, n, st.ux[i], st.uy[i], st.uz[i]);
  else if (kind == EV_DECAY && (!NUC || (c.A == 1 && c.Z == 0)))
    decay_event<NUC>(p, c);
  else if (kind == EV_DECAY)
    nuclear_decay<NUC>(p, st, dc, c, n, st.ux[i], st.uy[i], st.uz[i]);
  else
    reset_states<NUC>(p, c);
  st.E[i] = c.E;
  st.A[i] = c.A;
  st.Z[i] = c.Z;
  st.d_pion[i] = c.d_pion;
  st.d_pd[i] = c.d_pd;
  st.d_dec[i] = c.d_dec;
  st.draws[i] = c.draws;
  st.events[i] = c.events;
  st.n_pion[i] = c.n_pion;
  st.n_pd[i] = c.n_pd;
  st.n_dropped[i] = c.n_dropped;
  st.flags[i] = c.flags;
  if (n.pion) atomicAdd(&dc->pion, (unsigned long long)n.pion);
  if (n.pd) atomicAdd(&dc->pd, (unsigned long long)n.pd);
  if (n.sec) atomicAdd(&dc->secondaries, (unsigned long long)n.sec);
  if (n.dropped) atomicAdd(&dc->dropped, (unsigned long long)n.dropped);
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

// ---------------------------------------------------------------------------
// Hot per-lane state.
// ---------------------------------------------------------------------------
struct LaneCore {
  uint32_t slot;
  int A, Z, q, status;
  double x[3];
  // d_pd holds the candidate's second stochastic free path: photodisintegration
  // for nuclei, beta decay for free neutrons (the other one is infinite);
  // d_nd the decay of an unstable nucleus (kernels built with a nuclide table
  // only)
  double E, s, s_max, h, d_pion, d_pd, d_nd;
  uint32_t dacc, drej;  // accepted steps / rejected trials since the last store
  uint32_t budget;      // accepted steps left before CRP_BUDGET
  int rejections;       // rejected trials of the current step
  bool crossed;         // this step's segment entered the observer sphere
};

struct LaneCounters {
  uint32_t acc, rej, detected, pending_acc;
};

__device__ __forceinline__ bool is_neutron(const LaneCore& c) { return c.A == 1 && c.Z == 0; }

// Is the lane's second free path (photodisintegration, or decay for a free
// neutron) an active module?
// Module flags of a kernel: the run-time flags, or (FIX != 0) a module list
// fixed at compile time, which lets the compiler drop the modules it leaves out.
template <uint32_t FIX>
__device__ __forceinline__ uint32_t mflags(const KParams& p) {
  return FIX ? FIX : p.flags;
}

template <uint32_t FIX = 0>
__device__ __forceinline__ bool second_on(const KParams& p, const LaneCore& c) {
  return (mflags<FIX>(p) & (is_neutron(c) ? CRP_DECAY : CRP_PHOTODIS)) != 0;
}

// Is the lane's third free path (decay of a nucleus) active?  Only kernels
// instantiated with NUC (launched when a nuclide table is in use) hold it.
template <bool NUC, uint32_t FIX = 0>
__device__ __forceinline__ bool nuc_on(const KParams& p, const LaneCore& c) {
  return NUC && (mflags<FIX>(p) & CRP_DECAY) != 0 && c.A >= 2;
}

template <bool NUC = false>
__device__ __forceinline__ void load_core(const KParams& p, const DevState& st, uint32_t i,
                                          LaneCore& c) {
  c.slot = i;
  c.x[0] = st.x[i];
  c.x[1] = st.y[i];
  c.x[2] = st.z[i];
  c.E = st.E[i];
  c.s = st.s[i];
  c.s_max = st.s_max[i];
  c.h = st.h[i];
  c.d_pion = st.d_pion[i];
  c.A = st.A[i];
  c.Z = st.Z[i];
  c.d_pd = is_neutron(c) ? st.d_dec[i] : st.d_pd[i];
  if (NUC) c.d_nd = c.A >= 2 ? st.d_dec[i] : (double)INFINITY;
  c.q = st.q[i];
  c.status = st.status[i];
  const uint64_t done = st.n_acc[i];
  const uint64_t left = done >= p.max_steps ? 0 : p.max_steps - done;
  c.budget = left > 0xffffffffull ? 0xffffffffu : (uint32_t)left;
  c.dacc = 0;
  c.drej = 0;
  c.rejections = 0;
  c.crossed = false;
}

template <bool NUC = false>
__device__ __forceinline__ void store_core(const DevState& st, LaneCore& c) {
  const uint32_t i = c.slot;
  st.x[i] = c.x[0];
  st.y[i] = c.x[1];
  st.z[i] = c.x[2];
  st.E[i] = c.E;
  st.s[i] = c.s;
  st.h[i] = c.h;
  st.d_pion[i] = c.d_pion;
  if (is_neutron(c))
    st.d_dec[i] = c.d_pd;
  else
    st.d_pd[i] = c.d_pd;
  if (NUC && c.A >= 2) st.d_dec[i] = c.d_nd;
  st.status[i] = c.status;
  st.n_acc[i] += c.dacc;
  st.n_rej[i] += c.drej;
  c.dacc = 0;
  c.drej = 0;
}

// Fields a rare path may change.
template <bool NUC = false>
__device__ __forceinline__ void reload_event_fields(const DevState& st, LaneCore& c) {
  const uint32_t i = c.slot;
  c.E = st.E[i];
  c.A = st.A[i];
  c.Z = st.Z[i];
  c.d_pion = st.d_pion[i];
  c.d_pd = is_neutron(c) ? st.d_dec[i] : st.d_pd[i];
  if (NUC) c.d_nd = c.A >= 2 ? st.d_dec[i] : (double)INFINITY;
}

// One accepted step done: step budget bookkeeping.
__device__ __forceinline__ void count_step(LaneCore& c, LaneCounters& lc) {
  c.dacc += 1;
  if (c.budget) c.budget -= 1;
  lc.acc += 1;
  lc.pending_acc += 1;
}

__device__ __forceinline__ void count_reject(LaneCore& c, LaneCounters& lc) {
  c.rejections += 1;
  c.drej += 1;
  lc.rej += 1;
}

// Per-thread stage storage in shared memory: slot k of this thread lives at
// base[k * stride], so a warp touching one slot hits 32 consecutive words.
// Slots 0..17: stage directions U[j][c]; 18..35: stage forces K[j][c].
template <class T>
struct StageStore {
  T* base;
  int stride;
  __device__ __forceinline__ T& u(int j, int c) { return base[(j * 3 + c) * stride]; }
  __device__ __forceinline__ T& k(int j, int c) { return base[(18 + j * 3 + c) * stride]; }
};
constexpr int kStageSlots = 36;

// Cash-Karp tableau in constant memory (uniform across a warp whose lanes
// all run the same stage), for the stage loop.
static __constant__ double c_a64[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {ck::a21, 0, 0, 0, 0, 0},
    {ck::a31, ck::a32, 0, 0, 0, 0},
    {ck::a41, ck::a42, ck::a43, 0, 0, 0},
    {ck::a51, ck::a52, ck::a53, ck::a54, 0, 0},
    {ck::a61, ck::a62, ck::a63, ck::a64, ck::a65, 0}};
static __constant__ float c_a32[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {(float)ck::a21, 0, 0, 0, 0, 0},
    {(float)ck::a31, (float)ck::a32, 0, 0, 0, 0},
    {(float)ck::a41, (float)ck::a42, (float)ck::a43, 0, 0, 0},
    {(float)ck::a51, (float)ck::a52, (float)ck::a53, (float)ck::a54, 0, 0},
    {(float)ck::a61, (float)ck::a62, (float)ck::a63, (float)ck::a64, (float)ck::a65, 0}};

// ---------------------------------------------------------------------------
// FP64 policy.  begin_step / trial / finish_step / breaks split the module
// cycle so that a warp advances one Cash-Karp trial per iteration; the
// arithmetic and its order are those of the reference formulation.
// ---------------------------------------------------------------------------
template <bool NUC>
struct PolicyFP64T {
  static constexpr uint32_t kFix = 0;  // run-time module flags
  static constexpr bool kNuc = NUC;    // nuclear decay as a third free path
  using Real = double;
  static constexpr bool kSharedStages = true;
  static constexpr size_t kSmemPerThread = kStageSlots * sizeof(double);
  struct Lane : LaneCore {
    double u[3];
    double cap_s, kappa, eps;
    double y5[6];
  };
  __device__ __forceinline__ static void init_lane(Lane&) {}

  __device__ __forceinline__ static void load(const KParams& p, const DevState& st, uint32_t i,
                                              Lane& c) {
    load_core<NUC>(p, st, i, c);
    c.u[0] = st.ux[i];
    c.u[1] = st.uy[i];
    c.u[2] = st.uz[i];
  }
  __device__ __forceinline__ static void store(const DevState& st, Lane& c) {
    store_core<NUC>(st, c);
    st.ux[c.slot] = c.u[0];
    st.uy[c.slot] = c.u[1];
    st.uz[c.slot] = c.u[2];
  }

  template <class NodeT>
  __device__ __forceinline__ static void force(const KParams& p, const double x[3],
                                               const double u[3], double kappa, double k[3]) {
    double B[3];
    field_fp64<NodeT>(p, x, B);
    const double cx = u[1] * B[2] - u[2] * B[1];
    const double cy = u[2] * B[0] - u[0] * B[2];
    const double cz = u[0] * B[1] - u[1] * B[0];
    k[0] = kappa * cx;
    k[1] = kappa * cy;
    k[2] = kappa * cz;
  }

  template <class NodeT>
  __device__ __forceinline__ static void begin_step(const KParams& p, Lane& c,
                                                    StageStore<double>& S) {
    double h = c.h;
    if (h > p.h_max) h = p.h_max;
    c.cap_s = c.s_max - c.s;
    if (c.cap_s < h) h = c.cap_s;
    if ((p.flags & CRP_PION) && c.d_pion < h) h = c.d_pion;
    if (second_on(p, c) && c.d_pd < h) h = c.d_pd;
    if (nuc_on<NUC>(p, c) && c.d_nd < h) h = c.d_nd;
    c.h = h;  // trial step of this step
    c.kappa = (double)(c.q * c.Z) * p.curv_k / c.E;
    double k[3];
    force<NodeT>(p, c.x, c.u, c.kappa, k);
    for (int i = 0; i < 3; ++i) {
      S.u(0, i) = c.u[i];
      S.k(0, i) = k[i];
    }
    c.rejections = 0;
  }

  // One Cash-Karp trial with step c.h.  Returns true when accepted.
  template <class NodeT>
  __device__ __forceinline__ static bool trial(const KParams& p, Lane& c, StageStore<double>& S,
                                               LaneCounters& lc) {
    using namespace ck;
    const double h = c.h;
#pragma unroll 1
    for (int j = 1; j < 6; ++j) {
      double xs[3], us[3];
      for (int i = 0; i < 3; ++i) {
        double sx = c_a64[j][0] * S.u(0, i);
        double su = c_a64[j][0] * S.k(0, i);
        for (int m = 1; m < j; ++m) {
          sx = sx + c_a64[j][m] * S.u(m, i);
          su = su + c_a64[j][m] * S.k(m, i);
        }
        xs[i] = c.x[i] + h * sx;
        us[i] = c.u[i] + h * su;
      }
      double k[3];
      force<NodeT>(p, xs, us, c.kappa, k);
      for (int i = 0; i < 3; ++i) {
        S.u(j, i) = us[i];
        S.k(j, i) = k[i];
      }
    }
    double err[3];
    for (int i = 0; i < 3; ++i) {
      c.y5[i] = c.x[i] + h * (w1 * S.u(0, i) + w3 * S.u(2, i) + w4 * S.u(3, i) + w6 * S.u(5, i));
      c.y5[3 + i] =
          c.u[i] + h * (w1 * S.k(0, i) + w3 * S.k(2, i) + w4 * S.k(3, i) + w6 * S.k(5, i));
      err[i] = h * (d1 * S.k(0, i) + d3 * S.k(2, i) + d4 * S.k(3, i) + d5 * S.k(4, i) +
                    d6 * S.k(5, i));
    }
    c.eps = sqrt(err[0] * err[0] + err[1] * err[1] + err[2] * err[2]) / p.tol;
    if (c.eps <= 1.0 || h <= p.h_min || c.rejections >= 64) return true;
    double fac = 0.95 / sqrt(sqrt(c.eps));
    if (fac < 0.1) fac = 0.1;
    double hn = h * fac;
    if (hn < p.h_min) hn = p.h_min;
    c.h = hn;
    count_reject(c, lc);
    return false;
  }

  // Accepted step: state update, continuous losses, free-path bookkeeping.
  // Returns the stochastic interaction that fires (EV_NONE if none).
  __device__ __forceinline__ static int finish_step(const KParams& p, Lane& c,
                                                    LaneCounters& lc) {
    const double h = c.h;
    const double x_old[3] = {c.x[0], c.x[1], c.x[2]};
    c.x[0] = c.y5[0];
    c.x[1] = c.y5[1];
    c.x[2] = c.y5[2];
    const double un = sqrt(c.y5[3] * c.y5[3] + c.y5[4] * c.y5[4] + c.y5[5] * c.y5[5]);
    const double inv = 1.0 / un;
    c.u[0] = c.y5[3] * inv;
    c.u[1] = c.y5[4] * inv;
    c.u[2] = c.y5[5] * inv;
    c.s = (h == c.cap_s) ? c.s_max : c.s + h;
    double grow = c.eps == 0.0 ? 5.0 : 0.95 / sqrt(sqrt(c.eps));
    if (grow > 5.0) grow = 5.0;
    double h_next = h * grow;
    if (h_next < p.h_min) h_next = p.h_min;
    if (h_next > p.h_max) h_next = p.h_max;
    c.h = h_next;
    count_step(c, lc);
    c.crossed = (p.flags & CRP_OBSERVER) && segment_enters(x_old, c.x, p.obs_c, p.obs_r);
    // continuous losses
    if (p.flags & (CRP_PAIR | CRP_ADIABATIC)) {
      double beta = 0.0;
      if (p.flags & CRP_PAIR) {
        const double bp = table_fp64(p, p.t_beta, series_log(c.E / ((double)c.A * MP_C2_EV)));
        beta = bp * (double)(c.Z * c.Z) / (double)c.A;
      }
      if (p.flags & CRP_ADIABATIC) beta = beta + p.beta_ad;
      c.E = c.E * (1.0 - beta * h);
    }
    // stochastic interactions: the first in module order whose free path ran out
    const bool pion_on = (p.flags & CRP_PION) != 0;
    const bool pd_on = second_on(p, c);
    const bool nd_on = nuc_on<NUC>(p, c);
    if (pion_on) c.d_pion = c.d_pion - h;
    if (pd_on) c.d_pd = c.d_pd - h;
    if (nd_on) c.d_nd = c.d_nd - h;
    if (pion_on && c.d_pion <= 0.0) return EV_PION;
    if (pd_on && c.d_pd <= 0.0) return is_neutron(c) ? EV_DECAY : EV_PD;
    if (nd_on && c.d_nd <= 0.0) return EV_DECAY;
    return EV_NONE;
  }

  // Break conditions in module order: minimum energy, trajectory length,
  // observer, border; then the per-candidate step budget.
  __device__ __forceinline__ static void breaks(const KParams& p, Lane& c, LaneCounters& lc) {
    if ((p.flags & CRP_EMIN) && c.E < p.e_min) {
      c.status = CRP_BELOW_EMIN;
    } else if (c.s >= c.s_max) {
      c.status = CRP_MAX_LENGTH;
    } else if (c.crossed) {
      c.status = CRP_DETECTED;
      lc.detected += 1;
    } else if (p.flags & CRP_BORDER) {
      const double dx = c.x[0] - p.border_c[0], dy = c.x[1] - p.border_c[1],
                   dz = c.x[2] - p.border_c[2];
      if (dx * dx + dy * dy + dz * dz >= p.border_r * p.border_r) c.status = CRP_AT_BORDER;
    }
    if (c.status == CRP_ACTIVE && c.budget == 0) c.status = CRP_BUDGET;
  }

  __device__ __forceinline__ static void after_event(const KParams&, const DevState& st,
                                                     Lane& c) {
    reload_event_fields<NUC>(st, c);
  }

  __device__ __forceinline__ static uint32_t key(const KParams& p, const Lane& c) {
    return key_of_position(p, c.x[0], c.x[1], c.x[2]);
  }

  // Mid-step suspension: c.h already holds the current trial step, and a
  // resumed step restarts from it with the same caps and the same first stage.
  __device__ __forceinline__ static void suspend(Lane&) {}
};

// ---------------------------------------------------------------------------
// Mixed policy: binary32 field, force and stages relative to the current
// grid cell; binary64 position, trajectory length, energy, free paths and
// error norm (decided in binary64 near the tolerance).  GAL adds the
// analytic galactic field.
// ---------------------------------------------------------------------------
enum : int { CAP_NONE = 0, CAP_S = 1, CAP_PION = 2, CAP_PD = 3, CAP_ND = 4 };

// Accepted steps between exact rebases of a lane's binary32 cell coordinates
// on its binary64 position (and folds of its binary32 energy losses).  Each
// step adds one binary32 rounding (<= 2^-24 of a cell) to the in-cell
// coordinates, so after 128 steps they are within about 10^-6 of a cell of
// the binary64 position.  A rebase is about twenty binary64 operations that
// only the rebasing lanes of a warp execute, so a shorter period spends the
// binary64 pipe on nearly empty warp instructions.  Slices are rounded up to
// multiples of this period, so the rebase points depend only on each
// candidate's step count.
constexpr int kRebasePeriod = CRP_MIXED_REBASE_STEPS;

template <bool GAL, bool GMF = false, uint32_t FIX = 0, bool NUC = false>
struct PolicyMixedT {
  static constexpr uint32_t kFix = FIX;  // compile-time module list (0: run-time flags)
  static constexpr bool kNuc = NUC;      // nuclear decay as a third free path
  // The cell index of a record gather in 32 bits (records exist only for grids
  // of fewer than 2^32 cells) or in 64.  Only a register-allocation choice:
  // measured per instantiation, 32 bits made the extragalactic list (+0.8 %)
  // and the galactic back-tracking (+2.9 %) faster but the list with
  // photodisintegration slower (-2.2 %, a 4 B spill), so the others keep 64.
  static constexpr bool kCell32 = GAL || FIX == kModsEgal;
  using Real = float;
  static constexpr bool kSharedStages = false;
  // per-lane cache of the last cell record gathered (6 float4, lane-interleaved)
  static constexpr int kCacheF4 = 6;
  static constexpr size_t kSmemPerThread = kCacheF4 * sizeof(float4);
  struct LaneGal {
    float gal[3];  // position relative to the galactic centre
  };
  struct LaneNoGal {};
  struct Lane : LaneCore, std::conditional<GAL, LaneGal, LaneNoGal>::type {
    float u[3];
    int cell[3];    // grid cell of the current position
    float frac[3];  // in-cell fraction (grid units)
    float hf;       // trial step of the current step
    float hn;       // proposed next step, in [h_min, h_max]
    float E_f;      // binary32 copy of the energy
    float kap, d_obs, d_bord, err2, dx[3], u5[3];
    float3 k1;      // force at the start of the step
    int cap, since_rebase;
    uint32_t cell_key;  // index of the cell record held in this lane's cache
    // binary32 lower bound of the distance to the next length cap (s_max,
    // pending free paths); the exact binary64 tests run only when it is
    // below two proposed steps ("near")
    float near_f;
    bool near;
    // energy losses since the last fold: E = E_fold * (1 - yl), yl in binary32
    float yl, E_fold_f;
  };

  __device__ __forceinline__ static void init_lane(Lane& c) { c.cell_key = 0xffffffffu; }

  // Cell and fraction from the binary64 position (exact rebase).
  __device__ __forceinline__ static void rebase(const KParams& p, Lane& c) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double r = (c.x[d] - p.f.origin[d]) * p.f.inv_spacing;
      const double fl = floor(r);
      c.frac[d] = (float)(r - fl);
      c.cell[d] = (int)wrap_fl(fl, p.f.n[d], p.f.mask[d]);
    }
    if constexpr (GAL) {
#pragma unroll
      for (int d = 0; d < 3; ++d) c.gal[d] = (float)(c.x[d] - p.gal_c[d]);
    }
    c.since_rebase = 0;
  }

  // Conservative distances to the observer and border spheres (binary64
  // once; then lowered by each step's length, so the exact binary64 test
  // runs only when a sphere can be reached in the coming step).
  __device__ __forceinline__ static void bounds(const KParams& p, Lane& c) {
    if (mflags<FIX>(p) & CRP_OBSERVER) {
      const double a = c.x[0] - p.obs_c[0], b = c.x[1] - p.obs_c[1], d = c.x[2] - p.obs_c[2];
      const double r = sqrt(a * a + b * b + d * d);
      c.d_obs = (float)((r - p.obs_r) * (1.0 - 1e-6));
    }
    if (mflags<FIX>(p) & CRP_BORDER) {
      const double a = c.x[0] - p.border_c[0], b = c.x[1] - p.border_c[1],
                   d = c.x[2] - p.border_c[2];
      const double r = sqrt(a * a + b * b + d * d);
      c.d_bord = (float)((p.border_r - r) * (1.0 - 1e-6));
    }
  }

  __device__ __forceinline__ static void load(const KParams& p, const DevState& st, uint32_t i,
                                              Lane& c) {
    load_core<NUC>(p, st, i, c);
    c.u[0] = (float)st.ux[i];
    c.u[1] = (float)st.uy[i];
    c.u[2] = (float)st.uz[i];
    c.hn = fminf(fmaxf((float)c.h, p.h_min_f), p.h_max_f);
    c.E_f = (float)c.E;
    c.E_fold_f = c.E_f;
    c.yl = 0.f;
    rebase(p, c);
    bounds(p, c);
    set_near(p, c);
  }

  // Lower bound (binary32, rounded down) of the distance to the nearest
  // length cap: the end of the trajectory or a pending free path.
  __device__ __forceinline__ static void set_near(const KParams& p, Lane& c) {
    double d = c.s_max - c.s;
    if ((mflags<FIX>(p) & CRP_PION) && c.d_pion < d) d = c.d_pion;
    if (second_on<FIX>(p, c) && c.d_pd < d) d = c.d_pd;
    if (nuc_on<NUC, FIX>(p, c) && c.d_nd < d) d = c.d_nd;
    c.near_f = __double2float_rd(d);
  }

  // Apply the losses accumulated since the last fold to the binary64 energy.
  __device__ __forceinline__ static void fold_energy(Lane& c) {
    if (c.yl != 0.f) {
      c.E = c.E * (1.0 - (double)c.yl);
      c.E_f = (float)c.E;
      c.E_fold_f = c.E_f;
      c.yl = 0.f;
    }
  }

  __device__ __forceinline__ static void store(const DevState& st, Lane& c) {
    fold_energy(c);
    c.h = (double)c.hn;
    store_core<NUC>(st, c);
    st.ux[c.slot] = (double)c.u[0];
    st.uy[c.slot] = (double)c.u[1];
    st.uz[c.slot] = (double)c.u[2];
  }

  // Field at the current position plus offset (ox, oy, oz) (length unit).
  template <class NodeT>
  __device__ __forceinline__ static float3 field(const KParams& p, Lane& c, float ox,
                                                 float oy, float oz) {
    const FieldView& f = p.f;
    const float rx = fmaf(ox, f.inv_spacing_f, c.frac[0]);
    const float ry = fmaf(oy, f.inv_spacing_f, c.frac[1]);
    const float rz = fmaf(oz, f.inv_spacing_f, c.frac[2]);
    // the offsets span fewer than 2^20 cells (checked on the host), so the
    // in-cell coordinates stay within floor_small's range
    float fx, fy, fz;
    const int jx = floor_small(rx, fx), jy = floor_small(ry, fy), jz = floor_small(rz, fz);
    const float tx = rx - fx, ty = ry - fy, tz = rz - fz;
    const int nx = (int)f.n[0], ny = (int)f.n[1], nz = (int)f.n[2];
    const int ix0 = wrap_int(c.cell[0] + jx, nx, (int)f.mask[0]);
    const int iy0 = wrap_int(c.cell[1] + jy, ny, (int)f.mask[1]);
    const int iz0 = wrap_int(c.cell[2] + jz, nz, (int)f.mask[2]);
    float3 B;
    if (std::is_same<NodeT, float4>::value && f.cells) {
      // one aligned 128-byte record: the cell's trilinear polynomial,
      // evaluated in Horner form (7 FMAs per component)
      const size_t cell =
          kCell32 ? (size_t)(((uint32_t)iz0 * (uint32_t)ny + (uint32_t)iy0) * (uint32_t)nx +
                             (uint32_t)ix0)
                  : ((size_t)iz0 * ny + (size_t)iy0) * nx + (size_t)ix0;
      float4 a0, a1, a2, a3, a4, a5;
      // consecutive stages and steps mostly stay in one cell: re-read the
      // record from this lane's shared-memory copy (conflict-free, 4
      // wavefronts per warp load) instead of a 32-line global gather
      float4* cache = reinterpret_cast<float4*>(crp_dyn_smem) + threadIdx.x;
      const int bs = blockDim.x;
      if ((uint32_t)cell != c.cell_key || !f.cache_ok) {
        const float4* r = f.cells + 8 * cell;
        a0 = __ldg(r);
        a1 = __ldg(r + 1);
        a2 = __ldg(r + 2);
        a3 = __ldg(r + 3);
        a4 = __ldg(r + 4);
        a5 = __ldg(r + 5);
        cache[0] = a0;
        cache[bs] = a1;
        cache[2 * bs] = a2;
        cache[3 * bs] = a3;
        cache[4 * bs] = a4;
        cache[5 * bs] = a5;
        c.cell_key = (uint32_t)cell;
      } else {
        a0 = cache[0];
        a1 = cache[bs];
        a2 = cache[2 * bs];
        a3 = cache[3 * bs];
        a4 = cache[4 * bs];
        a5 = cache[5 * bs];
      }
      // coefficient j of component d is float 3j + d of the record
      auto horner = [&](float c0, float c1, float c2, float c3, float c4, float c5, float c6,
                        float c7) {
        const float xy = fmaf(fmaf(c7, tz, c4), ty, fmaf(c5, tz, c1));
        const float y0 = fmaf(fmaf(c6, tz, c2), ty, fmaf(c3, tz, c0));
        return fmaf(xy, tx, y0);
      };
      B.x = horner(a0.x, a0.w, a1.z, a2.y, a3.x, a3.w, a4.z, a5.y);
      B.y = horner(a0.y, a1.x, a1.w, a2.z, a3.y, a4.x, a4.w, a5.z);
      B.z = horner(a0.z, a1.y, a2.x, a2.w, a3.z, a4.y, a5.x, a5.w);
    } else {
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
      B.x = lerp(lerp(lerp(v0.x, v1.x, tx), lerp(v2.x, v3.x, tx), ty),
                 lerp(lerp(v4.x, v5.x, tx), lerp(v6.x, v7.x, tx), ty), tz);
      B.y = lerp(lerp(lerp(v0.y, v1.y, tx), lerp(v2.y, v3.y, tx), ty),
                 lerp(lerp(v4.y, v5.y, tx), lerp(v6.y, v7.y, tx), ty), tz);
      B.z = lerp(lerp(lerp(v0.z, v1.z, tx), lerp(v2.z, v3.z, tx), ty),
                 lerp(lerp(v4.z, v5.z, tx), lerp(v6.z, v7.z, tx), ty), tz);
    }
    if constexpr (GAL) {
      const float gx = c.gal[0] + ox, gy = c.gal[1] + oy, gz = c.gal[2] + oz;
      if (mflags<FIX>(p) & CRP_GALACTIC) {
        const float3 G = galactic_f32(p, gx, gy, gz);
        B.x += G.x;
        B.y += G.y;
        B.z += G.z;
      }
      if constexpr (GMF) {
        if (mflags<FIX>(p) & CRP_GMF) {
          const float3 G = gmf_f32(p, gx, gy, gz);
          B.x += G.x;
          B.y += G.y;
          B.z += G.z;
        }
      }
    }
    return B;
  }

  __device__ __forceinline__ static float3 force(float kap, float ux, float uy, float uz,
                                                 float3 B) {
    return make_float3(kap * (uy * B.z - uz * B.y), kap * (uz * B.x - ux * B.z),
                       kap * (ux * B.y - uy * B.x));
  }

  template <class NodeT>
  __device__ __forceinline__ static void begin_step(const KParams& p, Lane& c,
                                                    StageStore<float>&) {
    c.cap = CAP_NONE;
    c.hf = c.hn;
    // near_f bounds every cap distance from below: at or above two proposed
    // steps no cap can bind, and the binary64 comparisons are skipped
    c.near = c.near_f < 2.f * c.hn;
    if (c.near) {
      double h = (double)c.hn;
      const double rem = c.s_max - c.s;
      if (rem < h) {
        h = rem;
        c.cap = CAP_S;
      }
      if ((mflags<FIX>(p) & CRP_PION) && c.d_pion < h) {
        h = c.d_pion;
        c.cap = CAP_PION;
      }
      if (second_on<FIX>(p, c) && c.d_pd < h) {
        h = c.d_pd;
        c.cap = CAP_PD;
      }
      if (nuc_on<NUC, FIX>(p, c) && c.d_nd < h) {
        h = c.d_nd;
        c.cap = CAP_ND;
      }
      if (c.cap != CAP_NONE) c.hf = (float)h;
    }
    c.kap = (float)(c.q * c.Z) * p.curv_k_f / c.E_f;
    c.k1 = force(c.kap, c.u[0], c.u[1], c.u[2], field<NodeT>(p, c, 0.f, 0.f, 0.f));
    c.rejections = 0;
  }

  // One Cash-Karp trial; the stage vectors stay in registers (stages
  // unrolled), the first stage's force is reused across rejections.
  template <class NodeT>
  __device__ __forceinline__ static bool trial(const KParams& p, Lane& c, StageStore<float>&,
                                               LaneCounters& lc) {
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
    const float h = c.hf, kap = c.kap;
    const float3 u1 = make_float3(c.u[0], c.u[1], c.u[2]);
    const float3 k1 = c.k1;
    auto comb = [](float a, float3 x, float b, float3 y) {
      return make_float3(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z));
    };
    auto madd = [](float a, float3 x, float3 y) {
      return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
    };
    auto stage = [&](float3 osum, float3 ksum, float3& u_out) {
      u_out = madd(h, ksum, u1);
      return force(kap, u_out.x, u_out.y, u_out.z,
                   field<NodeT>(p, c, h * osum.x, h * osum.y, h * osum.z));
    };
    float3 u2, u3, u4, u5, u6;
    const float3 k2 = stage(make_float3(A21 * u1.x, A21 * u1.y, A21 * u1.z),
                            make_float3(A21 * k1.x, A21 * k1.y, A21 * k1.z), u2);
    const float3 k3 = stage(comb(A31, u1, A32, u2), comb(A31, k1, A32, k2), u3);
    const float3 k4 = stage(madd(A43, u3, comb(A41, u1, A42, u2)),
                            madd(A43, k3, comb(A41, k1, A42, k2)), u4);
    const float3 k5 = stage(madd(A54, u4, madd(A53, u3, comb(A51, u1, A52, u2))),
                            madd(A54, k4, madd(A53, k3, comb(A51, k1, A52, k2))), u5);
    const float3 k6 =
        stage(madd(A65, u5, madd(A64, u4, madd(A63, u3, comb(A61, u1, A62, u2)))),
              madd(A65, k5, madd(A64, k4, madd(A63, k3, comb(A61, k1, A62, k2)))), u6);
    const float3 dsum = madd(W6, u6, madd(W4, u4, comb(W1, u1, W3, u3)));
    const float3 usum = madd(W6, k6, madd(W4, k4, comb(W1, k1, W3, k3)));
    const float3 esum = madd(D6, k6, madd(D5, k5, madd(D4, k4, comb(D1, k1, D3, k3))));
    c.dx[0] = h * dsum.x;
    c.dx[1] = h * dsum.y;
    c.dx[2] = h * dsum.z;
    c.u5[0] = fmaf(h, usum.x, u1.x);
    c.u5[1] = fmaf(h, usum.y, u1.y);
    c.u5[2] = fmaf(h, usum.z, u1.z);
    const float e[3] = {h * esum.x, h * esum.y, h * esum.z};
    // Error norm: the binary32 sum of squares is within a few ulp of the
    // binary64 one, so it decides acceptance exactly as binary64 does except
    // in a +-1e-5 band around the tolerance, where the binary64 norm decides.
    const float e2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    c.err2 = e2;
    bool accept;
    if (e2 < 0.99999f * p.tol2_f) {
      accept = true;
    } else if (e2 > 1.00001f * p.tol2_f) {
      accept = false;
    } else {
      const double d0 = e[0], d1 = e[1], d2 = e[2];
      accept = d0 * d0 + d1 * d1 + d2 * d2 <= p.tol2;
    }
    if (accept || h <= p.h_min_f || c.rejections >= 64) return true;
    float fac = 0.95f * rsqrtf(sqrtf(sqrtf(e2 * p.inv_tol2_f)));  // 0.95 eps^(-1/4)
    fac = fmaxf(fac, 0.1f);
    c.hf = fmaxf(h * fac, p.h_min_f);
    c.cap = CAP_NONE;
    count_reject(c, lc);
    return false;
  }

  __device__ __forceinline__ static int finish_step(const KParams& p, Lane& c,
                                                    LaneCounters& lc) {
    const float hf = c.hf;
    const double h = (double)hf;
    const double x_old[3] = {c.x[0], c.x[1], c.x[2]};
    c.x[0] = c.x[0] + (double)c.dx[0];
    c.x[1] = c.x[1] + (double)c.dx[1];
    c.x[2] = c.x[2] + (double)c.dx[2];
    const float inv = rsqrtf(c.u5[0] * c.u5[0] + c.u5[1] * c.u5[1] + c.u5[2] * c.u5[2]);
    c.u[0] = c.u5[0] * inv;
    c.u[1] = c.u5[1] * inv;
    c.u[2] = c.u5[2] * inv;
    c.s = c.cap == CAP_S ? c.s_max : c.s + h;
    float grow = 5.f;
    if (c.err2 > 0.f) grow = fminf(5.f, 0.95f * rsqrtf(sqrtf(sqrtf(c.err2 * p.inv_tol2_f))));
    c.hn = fminf(fmaxf(hf * grow, p.h_min_f), p.h_max_f);
    count_step(c, lc);
    // field-lookup coordinate: advance in binary32, exact rebase every 32 steps
    if (++c.since_rebase >= kRebasePeriod) {
      rebase(p, c);
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float r = fmaf(c.dx[d], p.f.inv_spacing_f, c.frac[d]);
        float fl;
        const int j = floor_small(r, fl);
        c.frac[d] = r - fl;
        c.cell[d] = wrap_int(c.cell[d] + j, (int)p.f.n[d], (int)p.f.mask[d]);
      }
      if constexpr (GAL) {
#pragma unroll
        for (int d = 0; d < 3; ++d) c.gal[d] += c.dx[d];
      }
    }
    // observer: exact binary64 segment test only when the sphere is in reach
    c.crossed = false;
    if (mflags<FIX>(p) & CRP_OBSERVER) {
      c.d_obs -= 1.01f * hf;
      if (c.d_obs <= 0.f) {
        c.crossed = segment_enters(x_old, c.x, p.obs_c, p.obs_r);
        if (!c.crossed) bounds(p, c);
      }
    }
    // continuous losses
    if (mflags<FIX>(p) & (CRP_PAIR | CRP_ADIABATIC)) {
      float beta = 0.f;
      if (mflags<FIX>(p) & CRP_PAIR) {
        const float g = c.E_f / ((float)c.A * (float)MP_C2_EV);
        const float bp = table_f32(p, p.t_beta_f, __logf(g));
        beta = bp * (float)(c.Z * c.Z) / (float)c.A;
      }
      if (mflags<FIX>(p) & CRP_ADIABATIC) beta += p.beta_ad_f;
      // (1 - yl)(1 - x) = 1 - (yl + x - x yl): yl stays small, so its binary32
      // rounding is tiny against the energy; folded into binary64 every 32
      // steps (with the rebase), at events and when the lane is stored
      const float x = beta * hf;
      c.yl = fmaf(-x, c.yl, c.yl + x);
      c.E_f = c.E_fold_f * (1.f - c.yl);
    }
    if (c.since_rebase == 0) fold_energy(c);
    // stochastic interactions (a free path can end only in a "near" step)
    const bool pion_on = (mflags<FIX>(p) & CRP_PION) != 0;
    const bool pd_on = second_on<FIX>(p, c);
    const bool nd_on = nuc_on<NUC, FIX>(p, c);
    if (pion_on) c.d_pion = c.cap == CAP_PION ? 0.0 : c.d_pion - h;
    if (pd_on) c.d_pd = c.cap == CAP_PD ? 0.0 : c.d_pd - h;
    if (nd_on) c.d_nd = c.cap == CAP_ND ? 0.0 : c.d_nd - h;
    c.near_f = __fsub_rd(c.near_f, hf);
    if (c.near) {
      if (pion_on && c.d_pion <= 0.0) return EV_PION;
      if (pd_on && c.d_pd <= 0.0) return is_neutron(c) ? EV_DECAY : EV_PD;
      if (nd_on && c.d_nd <= 0.0) return EV_DECAY;
    }
    return EV_NONE;
  }

  __device__ __forceinline__ static void breaks(const KParams& p, Lane& c, LaneCounters& lc) {
    // E_f is within 1e-6 of the energy, so the binary64 test runs only near E_min;
    // s reaches s_max only in a "near" step
    if ((mflags<FIX>(p) & CRP_EMIN) && c.E_f < p.e_min_guard_f && c.E * (1.0 - (double)c.yl) < p.e_min) {
      c.status = CRP_BELOW_EMIN;
    } else if (c.near && c.s >= c.s_max) {
      c.status = CRP_MAX_LENGTH;
    } else if (c.crossed) {
      c.status = CRP_DETECTED;
      lc.detected += 1;
    } else if (mflags<FIX>(p) & CRP_BORDER) {
      c.d_bord -= 1.01f * c.hf;
      if (c.d_bord <= 0.f) {
        const double dx = c.x[0] - p.border_c[0], dy = c.x[1] - p.border_c[1],
                     dz = c.x[2] - p.border_c[2];
        if (dx * dx + dy * dy + dz * dz >= p.border_r * p.border_r)
          c.status = CRP_AT_BORDER;
        else
          bounds(p, c);
      }
    }
    if (c.status == CRP_ACTIVE && c.budget == 0) c.status = CRP_BUDGET;
  }

  __device__ __forceinline__ static void after_event(const KParams& p, const DevState& st,
                                                     Lane& c) {
    reload_event_fields<NUC>(st, c);
    c.E_f = (float)c.E;
    c.E_fold_f = c.E_f;
    c.yl = 0.f;
    set_near(p, c);
  }

  __device__ __forceinline__ static void suspend(Lane& c) { c.hn = c.hf; }

  __device__ __forceinline__ static uint32_t key(const KParams& p, const Lane& c) {
    return brick_key(c.cell[0], c.cell[1], c.cell[2], p.key_shift);
  }
};

using PolicyMixed = PolicyMixedT<false>;
using PolicyMixedGal = PolicyMixedT<true>;         // analytic disk + halo
using PolicyMixedGmf = PolicyMixedT<true, true>;   // plus the multi-arm field
using PolicyFP64 = PolicyFP64T<false>;
// with a nuclide table: the decay of unstable nuclei as a third free path
using PolicyFP64Nuc = PolicyFP64T<true>;
using PolicyMixedNuc = PolicyMixedT<false, false, 0, true>;
using PolicyMixedGalNuc = PolicyMixedT<true, false, 0, true>;
using PolicyMixedGmfNuc = PolicyMixedT<true, true, 0, true>;


// ---------------------------------------------------------------------------
// Persistent driver: lanes take candidates from the round's work queue, run
// at most `slice` accepted steps on each (one Cash-Karp trial per loop
// iteration for the whole warp), then requeue still-active candidates for
// the next round and take the next one.
// ---------------------------------------------------------------------------
// THREADS (largest block) and MINB (resident blocks per SM the register
// allocation is sized for) form a launch variant: registers per thread are
// at most 65536 / (THREADS * MINB).
template <class Policy, class NodeT, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    propagate_kernel(const KParams p, const DevState st, DevCounters* dc) {
  using Real = typename Policy::Real;
  using Lane = typename Policy::Lane;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StageStore<Real> S{reinterpret_cast<Real*>(smem_raw) + threadIdx.x, (int)blockDim.x};
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = globaltimer_ns();
  const uint64_t n_in = p.n_in_dev ? *p.n_in_dev : p.n_in;
  Lane c;
  Policy::init_lane(c);
  LaneCounters lc = {0, 0, 0, 0};
  bool has = false, exhausted = false, in_step = false;
  uint32_t slice_steps = 0;
  int iter = 0;
  for (;;) {
    // hand free lanes the next queue entries (one atomic per warp)
    const bool need = !has && !exhausted;
    const unsigned m = __ballot_sync(FULL_MASK, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&dc->head, (unsigned long long)__popc(m));
      base = __shfl_sync(FULL_MASK, base, leader);
      if (need) {
        const unsigned long long mine = base + __popc(m & ((1u << lane) - 1u));
        if (mine < n_in) {
          const uint32_t slot = p.queue_in[mine];
          if (st.status[slot] == CRP_ACTIVE) {
            if ((mflags<Policy::kFix>(p) & (CRP_PION | CRP_PHOTODIS | CRP_DECAY)) &&
                !(st.flags[slot] & CF_STATES_DRAWN))
              slot_event<Policy::kNuc>(p, st, dc, slot, EV_DRAW);  // first free paths
            Policy::load(p, st, slot, c);
            has = true;
            in_step = false;
            slice_steps = 0;
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (__ballot_sync(FULL_MASK, has || !exhausted) == 0) break;
    if (has) {
      if (!in_step) {
        Policy::template begin_step<NodeT>(p, c, S);
        in_step = true;
      }
      if (Policy::template trial<NodeT>(p, c, S, lc)) {
        const int ev = Policy::finish_step(p, c, lc);
        if (ev != EV_NONE) {
          Policy::store(st, c);
          slot_event<Policy::kNuc>(p, st, dc, c.slot, ev);
          Policy::after_event(p, st, c);
        }
        Policy::breaks(p, c, lc);
        in_step = false;
        slice_steps += 1;
        if (c.status != CRP_ACTIVE) {
          Policy::store(st, c);
          has = false;
        } else if (slice_steps >= p.slice) {
          Policy::store(st, c);
          const unsigned long long qo = atomicAdd(&dc->q_out, 1ull);
          if (qo < p.capacity) {
            p.queue_out[qo] = c.slot;
            p.keys_out[qo] = p.queue_order == 1 ? Policy::key(p, c) : rigidity_key(c.E, c.Z);
          }
          has = false;
        }
      }
    }
    if ((++iter & 63) == 0 && (p.step_budget || p.deadline_ns)) {
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
        if (has) {
          if (in_step) Policy::suspend(c);
          Policy::store(st, c);  // still active: resumable
        }
        break;
      }
    }
  }
  // fold lane counters into the call's totals; every completed step evaluated
  // the force once at its start and five times per trial
  const bool budgeted = p.step_budget || p.deadline_ns;
  const unsigned acc_rem = __reduce_add_sync(FULL_MASK, budgeted ? lc.pending_acc : lc.acc);
  const unsigned acc = __reduce_add_sync(FULL_MASK, lc.acc);
  const unsigned rej = __reduce_add_sync(FULL_MASK, lc.rej);
  const unsigned det = __reduce_add_sync(FULL_MASK, lc.detected);
  if (lane == 0) {
    if (acc_rem) atomicAdd(&dc->acc, (unsigned long long)acc_rem);
    if (rej) atomicAdd(&dc->rej, (unsigned long long)rej);
    const unsigned long long rhs = 6ull * acc + 5ull * rej;
    if (rhs) atomicAdd(&dc->rhs, rhs);
    if (det) atomicAdd(&dc->detected, (unsigned long long)det);
  }
}

template <class Policy>
size_t smem_bytes(int block) {
  return Policy::kSmemPerThread * (size_t)block;
}

template <class Policy, int THREADS, int MINB>
cudaError_t launch_policy(const KParams& kp, const DevState& st, DevCounters* dc, int grid,
                          int block, cudaStream_t s) {
  const size_t sm = smem_bytes<Policy>(block);
  // shared memory for MINB resident blocks (plus the 1 KB the system
  // reserves per block); the rest of the unified L1 caches the gathers
  int dev = 0, max_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int carveout = -1;  // binary64 stages: driver default
  if (!Policy::kSharedStages && max_sm > 0) {
    const size_t need = (size_t)MINB * (sm + 1024);
    carveout = (int)((100 * need + max_sm - 1) / max_sm);
    if (carveout > 100) carveout = 100;
  }
  if (kp.f.dtype == CRP_F32) {
    auto k = propagate_kernel<Policy, float4, THREADS, MINB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    k<<<grid, block, sm, s>>>(kp, st, dc);
  } else {
    auto k = propagate_kernel<Policy, DNode, THREADS, MINB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    k<<<grid, block, sm, s>>>(kp, st, dc);
  }
  return cudaGetLastError();
}

template <class Policy, int THREADS, int MINB>
cudaError_t occupancy_policy(int dtype, int block, int* bps) {
  const size_t sm = smem_bytes<Policy>(block);
  if (dtype == CRP_F32) {
    auto k = propagate_kernel<Policy, float4, THREADS, MINB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, block, sm);
  }
  auto k = propagate_kernel<Policy, DNode, THREADS, MINB>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, block, sm);
}

}  // namespace crp
