// propagate_1d.cu -- 1D mode with cosmology (binary64; built with
// -fmad=false so every multiply and add is rounded separately, in the order
// written).
//
// A candidate moves along the line of sight toward the observer; its state
// is its redshift z (stored in x), energy, species and the remaining optical
// depths of the stochastic processes.  Flat Lambda-CDM,
// H(z) = H0 sqrt(Om (1+z)^3 + OL) per length unit.  One step lowers z by dz,
// the smallest of: dz_max; the step whose relative pair loss is loss_max; z
// itself; and, for each stochastic process, the step that uses up its
// optical depth (the event then happens at the end of the step).  The step's
// comoving length is dz / H(z - dz/2).  Pair loss (explicit, start-of-step
// rate) and the exact adiabatic factor (1+z')/(1+z) update the energy.  At
// redshift z the photon background is (1+z)^3 denser and (1+z) hotter, so
// per comoving length a rate is (1+z)^2 times its z = 0 table value at
// (1+z) Gamma; free-neutron decay is 1 / ((1+z) gamma c tau).  Events,
// secondaries and lineage ids follow the 3D module list.  Arrival at z = 0
// is status DETECTED.
#include <math.h>

#include "crp_internal.cuh"
#include "device_common.cuh"

namespace crp {
namespace {

struct Cand1d {
  uint64_t id;
  double z, E, s, s_max, tp, tpd, tdec;  // tp, tpd, tdec: optical depths
  int A, Z, q, status;
  uint32_t draws, events, n_pion, n_pd, n_dropped, flags, generation;
  uint64_t n_acc;
};

__device__ __forceinline__ double hubble(const K1dParams& p, double z) {
  const double a = 1.0 + z;
  return p.H0 * sqrt(p.omega_m * a * a * a + p.omega_l);
}

__device__ __forceinline__ double lookup(const K1dParams& p, const double* tab, double lng) {
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

__device__ __forceinline__ double draw(const K1dParams& p, Cand1d& c) {
  const Philox4 w = draw4(p.seed, TAG_INTERACTION, c.id, c.draws);
  c.draws += 1;
  return u01_open(w.v0, w.v1);
}

// optical depths in module order [pion, photodisintegration, decay]
__device__ __forceinline__ void reset(const K1dParams& p, Cand1d& c) {
  if (p.flags & CRP_PION) c.tp = -series_log(draw(p, c));
  if (p.flags & CRP_PHOTODIS) c.tpd = -series_log(draw(p, c));
  if (p.flags & CRP_DECAY) c.tdec = -series_log(draw(p, c));
  c.flags |= CF_STATES_DRAWN;
}

struct Rates {
  double beta, pion, pd, dec;
};

__device__ __forceinline__ Rates rates(const K1dParams& p, const Cand1d& c, double z) {
  Rates r = {0.0, 0.0, 0.0, 0.0};
  const double a = 1.0 + z;
  const double lng = series_log(a * (c.E / ((double)c.A * MP_C2_EV)));
  if (p.flags & CRP_PAIR) r.beta = a * a * lookup(p, p.t_beta, lng) * (double)(c.Z * c.Z) / (double)c.A;
  if (p.flags & CRP_PION) r.pion = a * a * (double)c.A * lookup(p, p.t_pion, lng);
  if ((p.flags & CRP_PHOTODIS) && c.A >= 2) r.pd = a * a * (double)c.A * lookup(p, p.t_gdr, lng);
  if ((p.flags & CRP_DECAY) && c.A == 1 && c.Z == 0) r.dec = 1.0 / (a * c.E * p.decay_k);
  return r;
}

// Single-nucleon emission (as in 3D); the nucleon joins the next round.
__device__ void emit_nucleon(const K1dParams& p, const DevState& st, DevCounters* dc,
                             uint64_t slot, Cand1d& c, uint32_t& n_sec, uint32_t& n_drop) {
  const double u = draw(p, c);
  bool proton = u < (double)c.Z / (double)c.A;
  const int Ad = c.A - 1;
  if (proton && Ad >= 2 && c.Z - 1 == 0) proton = false;
  if (!proton && Ad >= 2 && Ad - c.Z == 0) proton = true;
  const double En = c.E / (double)c.A;
  const double Ed = c.E * (double)Ad / (double)c.A;
  if (!(p.flags & CRP_EMIN) || En >= p.e_min) {
    const unsigned long long k = atomicAdd(&dc->tail, 1ull);
    if (k < p.capacity) {
      st.id[k] = lineage_id(c.id, c.events);
      st.parent[k] = c.id;
      st.x[k] = c.z;
      st.y[k] = 0.0;
      st.z[k] = 0.0;
      st.ux[k] = st.ux[slot];
      st.uy[k] = st.uy[slot];
      st.uz[k] = st.uz[slot];
      st.x0[k] = c.z;
      st.y0[k] = 0.0;
      st.z0[k] = 0.0;
      st.ux0[k] = st.ux[slot];
      st.uy0[k] = st.uy[slot];
      st.uz0[k] = st.uz[slot];
      st.E[k] = En;
      st.E0[k] = En;
      st.s[k] = c.s;
      st.s_max[k] = c.s_max;
      st.h[k] = 0.0;
      st.d_pion[k] = 0.0;
      st.d_pd[k] = 0.0;
      st.d_dec[k] = 0.0;
      st.A[k] = 1;
      st.Z[k] = proton ? 1 : 0;
      st.A0[k] = 1;
      st.Z0[k] = proton ? 1 : 0;
      st.q[k] = c.q;
      st.status[k] = CRP_ACTIVE;
      st.draws[k] = 0;
      st.events[k] = 0;
      st.generation[k] = c.generation + 1;
      st.n_pion[k] = 0;
      st.n_pd[k] = 0;
      st.n_dropped[k] = 0;
      st.flags[k] = 0;
      st.lens_pixel[k] = 0xffffffffu;
      st.n_acc[k] = 0;
      st.n_rej[k] = 0;
      const unsigned long long qo = atomicAdd(&dc->q_out, 1ull);
      if (qo < p.capacity) p.queue_out[qo] = (uint32_t)k;
      n_sec += 1;
    } else {
      atomicAdd(&dc->overflow, 1ull);
      atomicOr(&dc->error_word, ERR_QUEUE_FULL);
    }
  } else {
    c.n_dropped += 1;
    n_drop += 1;
  }
  c.A = Ad;
  c.Z = c.Z - (proton ? 1 : 0);
  c.E = Ed;
  c.n_pd += 1;
  c.events += 1;
}

__device__ void run(const K1dParams& p, const DevState& st, DevCounters* dc, uint64_t slot,
                    uint32_t (&cnt)[6]) {
  Cand1d c;
  c.id = st.id[slot];
  c.z = st.x[slot];
  c.E = st.E[slot];
  c.s = st.s[slot];
  c.s_max = st.s_max[slot];
  c.tp = st.d_pion[slot];
  c.tpd = st.d_pd[slot];
  c.tdec = st.d_dec[slot];
  c.A = st.A[slot];
  c.Z = st.Z[slot];
  c.q = st.q[slot];
  c.status = st.status[slot];
  c.draws = st.draws[slot];
  c.events = st.events[slot];
  c.n_pion = st.n_pion[slot];
  c.n_pd = st.n_pd[slot];
  c.n_dropped = st.n_dropped[slot];
  c.flags = st.flags[slot];
  c.generation = st.generation[slot];
  c.n_acc = st.n_acc[slot];
  const bool pion_on = (p.flags & CRP_PION) != 0;
  const bool pd_on = (p.flags & CRP_PHOTODIS) != 0;
  const bool dec_on = (p.flags & CRP_DECAY) != 0;
  uint32_t steps = 0;
  while (c.status == CRP_ACTIVE) {
    if ((pion_on || pd_on || dec_on) && !(c.flags & CF_STATES_DRAWN)) reset(p, c);
    const double z = c.z;
    const Rates r = rates(p, c, z);
    const double H = hubble(p, z);
    double dz = p.dz_max;
    int cap = 0;
    if (r.beta > 0.0 && p.loss_max * H / r.beta < dz) dz = p.loss_max * H / r.beta;
    if (z <= dz) {
      dz = z;
      cap = 1;
    }
    if (pion_on && r.pion > 0.0 && c.tp * H / r.pion < dz) {
      dz = c.tp * H / r.pion;
      cap = 2;
    }
    if (pd_on && r.pd > 0.0 && c.tpd * H / r.pd < dz) {
      dz = c.tpd * H / r.pd;
      cap = 3;
    }
    if (dec_on && r.dec > 0.0 && c.tdec * H / r.dec < dz) {
      dz = c.tdec * H / r.dec;
      cap = 4;
    }
    const double z1 = cap == 1 ? 0.0 : z - dz;
    const double h = dz / hubble(p, z - 0.5 * dz);
    if (p.flags & CRP_PAIR) c.E = c.E * (1.0 - r.beta * h);
    if (p.flags & CRP_ADIABATIC) c.E = c.E * ((1.0 + z1) / (1.0 + z));
    c.z = z1;
    c.s = c.s + h;
    c.n_acc += 1;
    steps += 1;
    if (pion_on) c.tp = cap == 2 ? 0.0 : c.tp - r.pion * h;
    if (pd_on) c.tpd = cap == 3 ? 0.0 : c.tpd - r.pd * h;
    if (dec_on) c.tdec = cap == 4 ? 0.0 : c.tdec - r.dec * h;
    if (pion_on && c.tp <= 0.0) {
      c.E = c.E - 0.2 * c.E / (double)c.A;
      c.n_pion += 1;
      c.events += 1;
      cnt[1] += 1;
      reset(p, c);
    } else if (pd_on && c.A >= 2 && c.tpd <= 0.0) {
      emit_nucleon(p, st, dc, slot, c, cnt[3], cnt[4]);
      cnt[2] += 1;
      reset(p, c);
    } else if (dec_on && c.A == 1 && c.Z == 0 && c.tdec <= 0.0) {
      c.Z = 1;
      c.E = c.E * (MP_C2_EV / MN_C2_EV);
      c.events += 1;
      reset(p, c);
    }
    if ((p.flags & CRP_EMIN) && c.E < p.e_min) {
      c.status = CRP_BELOW_EMIN;
    } else if (c.z <= 0.0) {
      c.status = CRP_DETECTED;
      cnt[5] += 1;
    }
    if (c.status == CRP_ACTIVE && c.n_acc >= p.max_steps) c.status = CRP_BUDGET;
  }
  cnt[0] += steps;
  st.x[slot] = c.z;
  st.E[slot] = c.E;
  st.s[slot] = c.s;
  st.d_pion[slot] = c.tp;
  st.d_pd[slot] = c.tpd;
  st.d_dec[slot] = c.tdec;
  st.A[slot] = c.A;
  st.Z[slot] = c.Z;
  st.status[slot] = c.status;
  st.draws[slot] = c.draws;
  st.events[slot] = c.events;
  st.n_pion[slot] = c.n_pion;
  st.n_pd[slot] = c.n_pd;
  st.n_dropped[slot] = c.n_dropped;
  st.flags[slot] = c.flags;
  st.n_acc[slot] = c.n_acc;
}

// Persistent: lanes take queue entries (one atomic per warp) and run each
// candidate to the end.
__global__ void __launch_bounds__(128) k_propagate_1d(const K1dParams p, const DevState st,
                                                      DevCounters* dc) {
  const int lane = threadIdx.x & 31;
  uint32_t cnt[6] = {0, 0, 0, 0, 0, 0};  // steps, pion, pd, secondaries, dropped, detected
  for (;;) {
    const unsigned m = __activemask();
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&dc->head, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    const unsigned long long mine = base + __popc(m & ((1u << lane) - 1u));
    if (mine >= p.n_in) break;
    const uint32_t slot = p.queue_in[mine];
    if (st.status[slot] == CRP_ACTIVE) run(p, st, dc, slot, cnt);
  }
  if (cnt[0]) atomicAdd(&dc->acc, (unsigned long long)cnt[0]);
  if (cnt[1]) atomicAdd(&dc->pion, (unsigned long long)cnt[1]);
  if (cnt[2]) atomicAdd(&dc->pd, (unsigned long long)cnt[2]);
  if (cnt[3]) atomicAdd(&dc->secondaries, (unsigned long long)cnt[3]);
  if (cnt[4]) atomicAdd(&dc->dropped, (unsigned long long)cnt[4]);
  if (cnt[5]) atomicAdd(&dc->detected, (unsigned long long)cnt[5]);
}

}  // namespace

cudaError_t launch_propagate_1d(const K1dParams& p, const DevState& st, DevCounters* dc, int grid,
                                int block, cudaStream_t s) {
  k_propagate_1d<<<grid, block, 0, s>>>(p, st, dc);
  return cudaGetLastError();
}

}  // namespace crp
