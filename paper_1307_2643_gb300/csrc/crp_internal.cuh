// crp_internal.cuh -- device-side data layout shared by the library's kernels.
//
// Candidate pool: structure of arrays in HBM, one slot per candidate
// (primaries first, secondaries appended).  Each array is 256-byte aligned so
// a warp touching 32 consecutive slots issues full 32-byte sectors.  A
// candidate's whole propagation state lives in its slot (CRPropa 3.0,
// Sect. 3: all propagation state is stored in the candidate), which is what
// lets any warp pick any candidate up, stop it and resume it later.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/crp.h"

namespace crp {

// Binary64 grid node: (Bx, By, Bz, 0), 32-byte aligned for two 16-byte loads.
struct __align__(32) DNode {
  double x, y, z, w;
};

// ---- error reporting (api.cu) -------------------------------------------
void set_error(const char* fmt, ...);
crp_status fail_cuda(cudaError_t e, const char* what);
void* dev_alloc(size_t bytes);
void dev_free(void* p);

// ---- kernel error-word bits ---------------------------------------------
enum : uint32_t {
  ERR_QUEUE_FULL = 1u << 0,
  ERR_BAD_CANDIDATE = 1u << 1,
  ERR_TRIAL_LIMIT = 1u << 2,
  ERR_ROUND_LIMIT = 1u << 3,
};

// Nuclide table entry: rest-frame lifetime [s] (infinite: stable), the
// cumulative branching fractions after beta-, beta+ and neutron emission, and
// the channel taken by a uniform at or past the last sum (proton emission if
// its fraction is non-zero, else the last channel with a non-zero fraction).
constexpr int kNucEntry = 5;

// per-candidate flag bits
enum : uint32_t {
  CF_STATES_DRAWN = 1u << 0,
};

struct DevState {
  uint64_t *id, *parent;
  double *x, *y, *z, *ux, *uy, *uz;
  double *E, *s, *s_max, *h, *d_pion, *d_pd, *d_dec;
  double *x0, *y0, *z0, *ux0, *uy0, *uz0, *E0;
  uint64_t *n_acc, *n_rej;
  int32_t *A, *Z, *q, *A0, *Z0, *status;
  uint32_t *draws, *events, *generation, *n_pion, *n_pd, *n_dropped, *flags, *lens_pixel;
};

// Device-resident counters of one propagate call.
struct DevCounters {
  unsigned long long head;         // next entry of the input work queue to hand out
  unsigned long long tail;         // pool size (secondaries appended atomically)
  unsigned long long q_out;        // entries written to the output work queue
  unsigned long long acc, rej, rhs, pion, pd, secondaries, dropped, overflow, detected;
  unsigned int error_word;
  unsigned int stop;               // set when the step budget or deadline ran out
  unsigned long long n_in;         // graph mode: entries of this round's input queue
  unsigned long long rounds;       // graph mode: rounds run
  unsigned long long lens_fallback;  // lens application: candidates left to binary64
};

struct FieldView {
  const void* data;                // float4 (F32) or DNode (F64) per node
  const float4* cells;             // F32: 8 float4 per cell (polynomial records), or null
  int cache_ok;                    // cell indices fit 32 bits (per-lane record cache usable)
  int64_t n[3];
  int64_t mask[3];                 // n-1 when n is a power of two, else -1
  double origin[3];
  double spacing, inv_spacing;
  float inv_spacing_f;
  int dtype;
};

// Multi-arm galactic field (CRP_GMF), converted once on the host: the
// binary64 constants the FP64 policy evaluates with (each computed by the
// same single expression as the model's definition states it), and binary32
// copies for the mixed policy.
struct GmfView {
  double arm_b[8];
  double d_arm[8];        // ln arm_rx[j] - ln arm_rx[0]
  double ln_r0;           // ln arm_rx[0]
  double tan_p, sin_p, cos_p, period;  // period = 2 pi tan p
  double ring_b, r_ring, r_in, r_out, h_disk, w_disk;
  double halo_bn, halo_bs, halo_rn, halo_rs, halo_wh, halo_z0;
  double x_b, tan_t, sin_t, cos_t, x_rc, x_r;
  double cut_in2, cut_out2;  // squared spherical cuts (0: none)
  float f_arm_b[8], f_d_arm[8];
  float f_ln_r0, f_tan_p, f_sin_p, f_cos_p, f_period, f_inv_period;
  float f_ring_b, f_r_ring, f_r_in, f_r_out, f_h_disk, f_m2_inv_w_disk;
  float f_halo_bn, f_halo_bs, f_halo_rn, f_halo_rs, f_m2_inv_halo_wh, f_inv_halo_z0;
  float f_x_b, f_inv_tan_t, f_sin_t, f_cos_t, f_x_rc, f_inv_x_r, f_q;
  float f_cut_in2, f_cut_out2;
};

struct KParams {
  FieldView f;
  GmfView gm;
  double tol, tol2, h_min, h_max, curv_k, beta_ad, e_min;
  float e_min_guard_f;  // binary32 E_min plus 1e-4: below it the exact test runs
  double decay_k;       // neutron decay length per eV: c tau_n / (m_n c^2) [length unit]
  double length_unit_m;  // metres per length unit (nuclear decay lengths)
  // unstable nuclei (CRP_DECAY with a nuclide table; null otherwise): kNucEntry
  // doubles per nuclide 0 <= Z <= A <= nuc_amax at A (A + 1) / 2 + Z
  const double* nuc_tab;
  int32_t nuc_amax;
  // binary32 copies for the mixed policy (converted once on the host)
  float tol2_f, inv_tol2_f, h_min_f, h_max_f, curv_k_f, beta_ad_f, tab_lg0_f, tab_inv_dlg_f;
  const float* t_beta_f;
  float gdisk_b, gsin, gcos, ginv_hz, grmin, grmax, ghalo_b, ghalo_z0, ghalo_inv2s2;
  uint32_t flags;
  uint64_t seed;
  const double* t_beta;
  const double* t_pion;
  const double* t_gdr;
  double tab_lg0, tab_inv_dlg;
  int64_t tab_n;
  double obs_c[3], obs_r;
  double border_c[3], border_r;
  double disk_b, sin_pitch, cos_pitch, disk_hz, disk_rmin, disk_rmax;
  double halo_b, halo_z0, halo_sigma;
  double gal_c[3];
  uint64_t max_steps;
  uint64_t step_budget;
  uint64_t deadline_ns;
  uint64_t capacity;
  // work queues of one round: pool indices of active candidates
  const uint32_t* queue_in;
  uint64_t n_in;
  const unsigned long long* n_in_dev;  // graph mode: n_in read from the device
  uint32_t* queue_out;
  uint32_t* keys_out;              // spatial brick key of each queue_out entry
  int key_shift[3];                // cell -> brick shift per axis (32 bricks per axis)
  int queue_order;                 // 0: rigidity key, 1: spatial brick key (see crp.h)
  uint32_t slice;                  // accepted steps per candidate per round
};

// 1D mode with cosmology (flat Lambda-CDM; lengths comoving; x holds the
// candidate's redshift): parameters of one round.
struct K1dParams {
  uint32_t flags;
  uint64_t seed;
  double e_min;
  double H0, omega_m, omega_l;  // H0 per length unit (H0 / c)
  double dz_max, loss_max;
  const double *t_beta, *t_pion, *t_gdr;
  double tab_lg0, tab_inv_dlg;
  int64_t tab_n;
  double decay_k;
  uint64_t capacity, max_steps;
  const uint32_t* queue_in;
  uint64_t n_in;
  uint32_t* queue_out;
};
cudaError_t launch_propagate_1d(const K1dParams& p, const DevState& st, DevCounters* dc, int grid,
                                int block, cudaStream_t s);

// Launch one propagate round over the candidates listed in kp.queue_in.
cudaError_t launch_propagate_fp64(const KParams& kp, const DevState& st, DevCounters* dc,
                                  int grid, int block, cudaStream_t s);
cudaError_t launch_propagate_mixed(const KParams& kp, const DevState& st, DevCounters* dc,
                                   int grid, int block, int variant, cudaStream_t s);
cudaError_t occupancy_propagate_fp64(int dtype, int block, int* blocks_per_sm, bool nuc);
// Kernels with the decay of unstable nuclei as a third free path (a nuclide
// table is in use); the mixed ones in the 256 x 2 launch variant only.
cudaError_t launch_propagate_fp64_nuc(const KParams& kp, const DevState& st, DevCounters* dc,
                                      int grid, int block, cudaStream_t s);
cudaError_t occupancy_propagate_fp64_nuc(int dtype, int block, int* blocks_per_sm);
cudaError_t launch_propagate_mixed_nuc(const KParams& kp, const DevState& st, DevCounters* dc,
                                       int grid, int block, cudaStream_t s);
cudaError_t occupancy_propagate_mixed_nuc(int dtype, uint32_t flags, int block, int* bps);
// Module lists the mixed kernel is also instantiated for with the list fixed
// at compile time (launch variant 256 x 2): extragalactic propagation with or
// without photodisintegration.
constexpr uint32_t kModsEgal = CRP_PAIR | CRP_ADIABATIC | CRP_PION | CRP_EMIN | CRP_OBSERVER;
constexpr uint32_t kModsEgalPd = kModsEgal | CRP_PHOTODIS;
constexpr uint32_t kModsGalBorder = CRP_GALACTIC | CRP_BORDER;  // galactic back-tracking
constexpr uint32_t kModsGmfBorder = CRP_GMF | CRP_BORDER;  // multi-arm back-tracking
int fixed_modules_index(uint32_t flags);  // -1: no fixed instantiation
cudaError_t launch_propagate_mixed_fixed(int index, const KParams& kp, const DevState& st,
                                         DevCounters* dc, int grid, int block, cudaStream_t s);
cudaError_t occupancy_propagate_mixed_fixed(int index, int dtype, int block, int* bps);
cudaError_t launch_propagate_mixed_gmf(const KParams& kp, const DevState& st, DevCounters* dc,
                                       int grid, int block, int variant, cudaStream_t s);
cudaError_t occupancy_propagate_mixed_gmf(int dtype, uint32_t flags, int variant, int block,
                                          int* bps);
cudaError_t sample_field_mixed_gmf(const KParams& kp, const double* xyz, int64_t n, double* B,
                                   cudaStream_t s);
cudaError_t occupancy_propagate_mixed(int dtype, uint32_t flags, int variant, int block,
                                      int* blocks_per_sm, bool nuc);
// Dynamic shared memory of one propagate block (per-thread stage storage).
size_t propagate_smem_fp64(int block);
// The field the propagate kernels see, at n points (device arrays xyz [n][3]
// and B [n][3], binary64): the binary64 path's interpolation, or the mixed
// path's (binary32, from the position's cell and fraction).
cudaError_t sample_field_fp64(const KParams& kp, const double* xyz, int64_t n, double* B,
                              cudaStream_t s);
cudaError_t sample_field_mixed(const KParams& kp, const double* xyz, int64_t n, double* B,
                               cudaStream_t s);
size_t propagate_smem_mixed(int block);

}  // namespace crp
