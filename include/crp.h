/*
 * crp.h -- C ABI of the GB300 candidate propagator.
 *
 * The library advances many independent cosmic-ray candidates (protons and
 * nuclei) through a gridded magnetic field, following the module / candidate
 * / IsActive statement of the propagation problem in CRPropa 3.0
 * (Alves Batista et al., ICRC 2013, arXiv:1307.2643, Sect. 3 and Fig. 1):
 *   - a candidate holds all of its propagation state, so candidates are
 *     processed concurrently (Sect. 3, "Cosmic Ray Candidate and Modules");
 *   - per step the module list runs in order: integration (deflection in the
 *     field; updates position, direction and trajectory length), interaction
 *     modules (continuous losses; stochastic interactions that decide
 *     independently and reset all interaction states after any interaction),
 *     boundary and observer modules; IsActive is checked after each cycle;
 *   - interactions append secondary candidates (Sect. 3).
 *
 * Conventions for every call:
 *   - Every call returns a crp_status; 0 is success, negative values are
 *     errors.  crp_last_error() returns a message for the calling thread's
 *     last failure.  No call aborts, traps or waits without a bound.
 *   - Pointers marked "host" are CPU memory, "device" are CUDA device memory
 *     of the context's device.  The library never keeps a caller's pointer
 *     after a call returns; caller buffers stay owned by the caller.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return data to the host synchronise that stream.
 *   - All device memory the library uses is owned by the context (or by the
 *     grid / tables / lens object) and released by the matching destroy
 *     call.  It is taken from crp_set_allocator's functions when set, else
 *     from cudaMalloc / cudaFree.
 *   - Results are a pure function of (seed, injected arrays, grid, tables,
 *     modules): they do not depend on the launch configuration.
 */
#ifndef CRP_H_
#define CRP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t crp_status;
#define CRP_OK 0
#define CRP_E_INVALID (-1)     /* bad argument; nothing was changed        */
#define CRP_E_OOM (-2)         /* device allocation failed                 */
#define CRP_E_CUDA (-3)        /* a CUDA runtime / cuFFT call failed       */
#define CRP_E_QUEUE_FULL (-4)  /* secondaries did not fit the capacity     */
#define CRP_E_TIMEOUT (-5)     /* step budget or deadline reached; resumable */
#define CRP_E_BOUNDS (-6)      /* a kernel index check failed (error word) */
#define CRP_E_STATE (-7)       /* call not valid in the context's state    */

typedef struct crp_context crp_context;
typedef struct crp_grid crp_grid;
typedef struct crp_tables crp_tables;
typedef struct crp_lens crp_lens;
typedef struct crp_mlp crp_mlp;

/* Message describing the calling thread's last failed call ("" if none). */
const char* crp_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t crp_version(void);

/* ------------------------------------------------------------------------
 * Device memory.  Optional allocator used by every later allocation of the
 * process (for instance a framework's caching allocator).  alloc returns a
 * device pointer of at least `bytes` bytes aligned to 256 bytes, or NULL.
 * Pass NULL functions to return to cudaMalloc / cudaFree.  Objects must be
 * destroyed with the allocator that created them still installed.
 * ---------------------------------------------------------------------- */
typedef void* (*crp_alloc_fn)(size_t bytes, void* user);
typedef void (*crp_free_fn)(void* ptr, void* user);
crp_status crp_set_allocator(crp_alloc_fn alloc, crp_free_fn release, void* user);

/* ------------------------------------------------------------------------
 * Context: one device, one random seed, one candidate pool of fixed
 * capacity (primaries plus all secondaries they may spawn).  The pool is
 * the set of candidates of the paper's Sect. 3; each candidate's record is
 * self-contained.  Device memory is taken on the first inject.
 * ---------------------------------------------------------------------- */
crp_status crp_context_create(int32_t device, uint64_t seed, size_t capacity, crp_context** out);
crp_status crp_context_destroy(crp_context* ctx);
/* Number of candidates in the pool (primaries + secondaries so far). */
crp_status crp_context_size(const crp_context* ctx, size_t* n_out);

/* ------------------------------------------------------------------------
 * Field grid (Sect. 4, "Magnetic field techniques": precomputed fields on
 * grids for fast lookup).  Vertex-centred and periodic: node (i, j, k) sits
 * at origin + (i, j, k) * spacing and index i wraps modulo n[0]; the field
 * between nodes is the trilinear interpolation, along x, then y, then z.
 * Units are the caller's: lengths in `length unit`, field in `field unit`
 * (crp_modules names both).
 * ---------------------------------------------------------------------- */
#define CRP_F32 0
#define CRP_F64 1

#define CRP_GRID_FROM_HOST 0    /* copy `data` from host memory            */
#define CRP_GRID_FROM_DEVICE 1  /* copy `data` from device memory          */
#define CRP_GRID_TURBULENT 2    /* generate a Kolmogorov turbulent field    */

typedef struct {
  int64_t n[3];          /* nodes along x, y, z (each >= 2)                  */
  double spacing;        /* node spacing (length unit), > 0                  */
  double origin[3];      /* position of node (0, 0, 0)                       */
  int32_t dtype;         /* storage / interpolation type: CRP_F32 | CRP_F64 */
  int32_t source;        /* CRP_GRID_*                                       */
  /* FROM_HOST / FROM_DEVICE: field values, layout [n2][n1][n0][3]
   * (x fastest, components Bx, By, Bz adjacent), element type data_dtype.  */
  const void* data;
  int32_t data_dtype;
  /* F32 grids: 0 = also store, per cell, its 8 corner vectors in one aligned
   * 128-byte record (24 floats; 8x the node array), so that the mixed
   * path's trilinear gather reads one cache line; -1 = nodes only.  When the
   * records do not fit in memory the grid is created without them. */
  int32_t cell_records;
  /* TURBULENT: Gaussian Fourier modes with 2pi/lmax <= |k| <= 2pi/lmin,
   * projected perpendicular to k (divergence free), power |B(k)|^2 ~ |k|^index
   * (index = -11/3 for Kolmogorov), inverse FFT, real part, mean removed,
   * scaled so that <|B|^2> = brms^2.  Modes on a Nyquist plane stay empty.
   * Random numbers: Philox4x32-10, key = seed, counter = (component, 1,
   * mode index lo, mode index hi), Box-Muller on two uniforms per component.  */
  double lmin, lmax, brms, spectral_index;
  uint64_t seed;
} crp_grid_desc;

crp_status crp_grid_create(crp_context* ctx, const crp_grid_desc* desc, crp_grid** out);
crp_status crp_grid_destroy(crp_grid* grid);
/* Copy the stored field to host memory as float64, layout [n2][n1][n0][3]. */
crp_status crp_grid_copy_out(const crp_grid* grid, double* host_out);

/* ------------------------------------------------------------------------
 * Interaction tables (Sect. 2 interactions; the paper gives no formulas).
 * n nodes uniform in ln(Gamma) over [gamma_lo, gamma_hi], values in
 * 1 / length unit, linear interpolation in ln(Gamma), clamped at both ends:
 *   beta_pair[i]: (1/E) dE/dx of a proton by pair production on a blackbody
 *     of temperature T_cmb, from Blumenthal, Phys. Rev. D 1, 1596 (1970)
 *     with the phi(kappa) fit of Chodorowski, Zdziarski & Sikora, ApJ 400,
 *     181 (1992); a nucleus (A, Z) loses (Z^2 / A) beta_pair(Gamma).  With
 *     irb_dilution[k] > 0 the background also holds a synthetic infrared /
 *     optical light of dilute blackbodies (temperature irb_T_K[k], photon
 *     density irb_dilution[k] times Planck's); the loss is linear in the
 *     photon density, so each adds irb_dilution[k] times the blackbody beta
 *     at irb_T_K[k].
 *   rate_pion[i]: photo-pion rate of one nucleon for a step cross section
 *     pion_sigma above the rest-frame photon energy pion_eth; a nucleus has
 *     A times that rate.
 *   rate_gdr[i]: photodisintegration rate per nucleon for a Lorentzian giant
 *     dipole resonance (peak gdr_peak per nucleon at gdr_center, full width
 *     gdr_fwhm, cut to [gdr_lo, gdr_hi]); a nucleus with A >= 2 has A times it.
 * ---------------------------------------------------------------------- */
typedef struct {
  int64_t n;                 /* >= 2 */
  double gamma_lo, gamma_hi; /* Lorentz-factor range, 0 < lo < hi */
  double length_unit_m;      /* metres per length unit */
  double T_cmb;              /* blackbody temperature [K] */
  double pion_sigma_mb, pion_eth_eV;
  double gdr_peak_mb, gdr_center_eV, gdr_fwhm_eV, gdr_lo_eV, gdr_hi_eV;
  double irb_T_K[2];         /* synthetic infrared / optical components [K] */
  double irb_dilution[2];    /* their dilution factors (0 = absent) */
} crp_tables_desc;

/* Compute the tables on the device (quadrature kernels). */
crp_status crp_tables_build(crp_context* ctx, const crp_tables_desc* desc, crp_tables** out);
/* Use tables supplied by the caller (host arrays of desc->n doubles each). */
crp_status crp_tables_from_host(crp_context* ctx, const crp_tables_desc* desc,
                                const double* beta_pair, const double* rate_pion,
                                const double* rate_gdr, crp_tables** out);
crp_status crp_tables_copy_out(const crp_tables* t, double* beta_pair, double* rate_pion,
                               double* rate_gdr);
crp_status crp_tables_destroy(crp_tables* t);

/* Decay of unstable nuclei (Sect. 2 lists nuclear decay among the
 * interactions; the paper gives no table).  Attaches a nuclide table to t:
 * n host entries (A[i], Z[i]), 2 <= A <= CRP_DECAY_MAX_A, 1 <= Z <= A - 1,
 * each listed once, with the rest-frame mean lifetime tau_s[i] > 0 [s] and
 * the branching fractions branching[4 i + k] >= 0 of k = 0 beta- (Z + 1),
 * 1 beta+ (Z - 1), 2 neutron emission (A - 1), 3 proton emission (A - 1,
 * Z - 1), summing to 1 within 1e-9; a channel with a non-zero fraction
 * whose daughter would have Z' = 0 or N' = 0 with A' >= 2 is rejected
 * (CRP_E_INVALID, the table unchanged).  Nuclides not listed are stable.
 * n = 0 removes the table.  The caller keeps its arrays; synchronous.
 * With CRP_DECAY in the modules and this table present, crp_propagate
 * decays the listed nuclei as a stochastic state reset with the others: the
 * free path is -ln(u) gamma c tau with gamma = E / (A m_p c^2); at the event
 * one uniform picks the channel as the first whose cumulative fraction (in
 * the order above) exceeds it, else the last channel with a non-zero
 * fraction; beta decays keep the energy (mass A m_p; the leptons are not
 * followed), nucleon emission gives the nucleon E / A and the daughter
 * E (A - 1) / A and appends the nucleon as a secondary (like
 * photodisintegration).  The 1D mode rejects such tables with CRP_DECAY. */
#define CRP_DECAY_MAX_A 64
crp_status crp_tables_set_decay(crp_tables* t, int64_t n, const int32_t* A, const int32_t* Z,
                                const double* tau_s, const double* branching);

/* ------------------------------------------------------------------------
 * Candidates (Sect. 3, source model: position, spectrum, composition).
 * Structure of arrays, n entries each, host or device memory (on_device).
 * Appended to the pool; ids are id[i], or first_id + i when id is NULL.
 * Directions must be unit vectors.  A >= 1, 0 <= Z <= A.
 * ---------------------------------------------------------------------- */
/* Accepted steps between the mixed path's exact rebases of a candidate's
 * binary32 cell coordinates on its binary64 position. */
#define CRP_MIXED_REBASE_STEPS 128

typedef struct {
  const uint64_t* id;                        /* optional */
  const double *x, *y, *z;                   /* position (length unit)   */
  const double *ux, *uy, *uz;                /* unit direction           */
  const double* E;                           /* energy [eV], > 0         */
  const int32_t *A, *Z;                      /* mass and charge numbers  */
  const int32_t* q;                          /* optional charge sign +1/-1 (antiparticles -1) */
  const double* s_max;                       /* optional trajectory budget (default +inf) */
  int32_t on_device;                         /* 1: device pointers, 0: host */
  int32_t reserved;
} crp_candidate_arrays;

crp_status crp_candidates_inject(crp_context* ctx, const crp_candidate_arrays* a, size_t n,
                                 uint64_t first_id, void* stream);
/* Empty the pool (keeps its memory). */
crp_status crp_candidates_clear(crp_context* ctx);

/* ------------------------------------------------------------------------
 * Module list and propagation.
 * ---------------------------------------------------------------------- */
#define CRP_FP64 0   /* every step in float64                                    */
#define CRP_MIXED 1  /* field, Lorentz force, RK stages float32; positions,
                        trajectory length, energy, free paths and the
                        step-error norm float64                                 */

/* module flags */
#define CRP_PAIR (1u << 0)       /* pair production on the CMB (continuous)   */
#define CRP_ADIABATIC (1u << 1)  /* adiabatic loss beta_ad (continuous)       */
#define CRP_PION (1u << 2)       /* photo-pion production (stochastic)        */
#define CRP_PHOTODIS (1u << 3)   /* photodisintegration (stochastic, secondaries) */
#define CRP_EMIN (1u << 4)       /* break below e_min                         */
#define CRP_OBSERVER (1u << 5)   /* observer sphere: detect on entry          */
#define CRP_BORDER (1u << 6)     /* border sphere: stop on reaching it        */
#define CRP_GALACTIC (1u << 7)   /* add the analytic galactic disk+halo field */
/* free-neutron beta decay (stochastic, after photodisintegration in module
 * order): a neutron (A = 1, Z = 0) decays after -ln(u) gamma c tau_n
 * (tau_n = 878.4 s, gamma = E / m_n c^2) into a proton of the same Lorentz
 * factor (E <- E m_p / m_n); every reset of the interaction states then
 * draws one more uniform, for every species */
#define CRP_DECAY (1u << 8)
/* add the analytic multi-arm galactic field of m->gmf (crp_gmf, below) */
#define CRP_GMF (1u << 9)

/* Analytic multi-arm galactic field of the Jansson-Farrar class (Sect. 4
 * names analytic galactic field models, JF12 among them; the structure is
 * that of R. Jansson and G. R. Farrar, ApJ 757:14, 2012, and the parameter
 * values are the caller's).  Galactocentric cylindrical (r, phi, z) about
 * m->gal_center, phi = atan2(y, x); lengths and fields in the units of
 * crp_modules.  L(t, h, w) = 1 / (1 + exp(-2 (|t| - h) / w)).
 *  disk, times (1 - L(z, h_disk, w_disk)):
 *    r_ring <= r < r_in:  B = ring_b phi_hat (ring);
 *    r_in <= r <= r_out:  B = arm_b[j] (r_in / r) (sin p r_hat + cos p phi_hat),
 *      j = the arm holding the logarithmic spiral (d ln r / d phi = tan p)
 *      through the point: the spiral crosses phi = pi at
 *      ln r_x = ln r + (pi - phi) tan p (modulo 2 pi tan p), and arm j holds
 *      r_x in [arm_rx[j], arm_rx[j+1]), arm_rx[8] = arm_rx[0] e^{2 pi tan p}.
 *      Divergence-free when sum_j arm_b[j] ln(arm_rx[j+1] / arm_rx[j]) = 0.
 *  toroidal halo: B_phi = e^{-|z|/halo_z0} L(z, h_disk, w_disk) times
 *    halo_bn (1 - L(r, halo_rn, halo_wh)) for z >= 0, halo_bs (1 - L(r, halo_rs,
 *    halo_wh)) for z < 0.
 *  X field: straight lines in the (r, z) plane crossing the midplane at r_p
 *    with strength x_b e^{-r_p / x_r} there, flux conserved along each line.
 *    Where r_p = r - |z| / tan x_theta >= x_rc: elevation x_theta,
 *    |B| = x_b e^{-r_p/x_r} r_p / r.  Elsewhere r_p = r f, f = x_rc / (x_rc +
 *    |z| / tan x_theta), elevation atan(x_rc tan x_theta / r_p),
 *    |B| = x_b e^{-r_p/x_r} f^2.  B_z = |B| sin(elev.), B_r = sign(z) |B| cos(elev.).
 *  zero inside the sphere r_cut_in and outside r_cut_out (0: no cut); on the
 *  axis r = 0 only B_z remains.
 * Requirements (else CRP_E_INVALID): 0 < arm_rx[0] < ... < arm_rx[7] <
 * arm_rx[0] e^{2 pi tan p}; 0 < |pitch_rad| < pi/2; w_disk, halo_wh, halo_z0 > 0;
 * r_in > 0; if x_b != 0: 0 < x_theta_rad < pi/2, x_rc > 0, x_r > 0.
 * The binary64 path evaluates every transcendental with the library's own
 * series (logarithm, exponential, arctangent by argument halving), so its
 * field is reproducible bit for bit. */
typedef struct {
  double arm_b[8];       /* arm strengths at r = r_in (field units) */
  double arm_rx[8];      /* arm boundary radii on the phi = pi ray, ascending */
  double pitch_rad;      /* spiral pitch p */
  double ring_b;         /* ring field (r_ring <= r < r_in) */
  double r_ring, r_in, r_out;
  double h_disk, w_disk; /* disk / halo transition height and width */
  double halo_bn, halo_bs, halo_rn, halo_rs, halo_wh, halo_z0;
  double x_b, x_theta_rad, x_rc, x_r;
  double r_cut_in, r_cut_out;
} crp_gmf;

typedef struct {
  int32_t precision;         /* CRP_FP64 | CRP_MIXED */
  uint32_t flags;            /* CRP_PAIR | ... */
  double tol;                /* Cash-Karp tolerance on the direction error */
  double h_min, h_max;       /* step bounds (length unit) */
  double field_unit_T;       /* tesla per field unit (1e-13 for nG) */
  double length_unit_m;      /* metres per length unit (Mpc: 3.0856775814913673e22) */
  double beta_ad;            /* adiabatic loss rate (1 / length unit) */
  double e_min;              /* [eV] */
  const crp_tables* tables;  /* required by PAIR / PION / PHOTODIS */
  double observer_center[3], observer_radius;
  double border_center[3], border_radius;
  /* analytic galactic field (CRP_GALACTIC), in field / length units:
   * disk  B = disk_b exp(-|z|/disk_hz) (sin p r_hat + cos p phi_hat) for
   *       disk_rmin <= r <= disk_rmax, p = disk_pitch_rad;
   * halo  B_phi = halo_b sign(z) exp(-(|z| - halo_z0)^2 / (2 halo_sigma^2)),
   * cylindrical coordinates about gal_center. */
  double disk_b, disk_pitch_rad, disk_hz, disk_rmin, disk_rmax;
  double halo_b, halo_z0, halo_sigma;
  double gal_center[3];
  uint64_t max_steps;        /* per-candidate accepted-step budget; 0 = 1e8.  A
                                candidate reaching it stops with CRP_BUDGET. */
  uint64_t step_budget;      /* accepted steps in this call before TIMEOUT (0 = none) */
  double deadline_ms;        /* wall-clock limit of this call (0 = none) */
  int32_t block_size;        /* threads per block, multiple of 32, at most 128 (FP64)
                                or 256 (MIXED); 0 = that maximum */
  int32_t blocks_per_sm;     /* resident blocks per SM (0 = occupancy maximum) */
  uint32_t slice;            /* accepted steps a lane runs on one candidate before
                                requeueing it for the next round (0 = 2^20: in
                                practice to the end); the mixed path rounds it up
                                to a multiple of CRP_MIXED_REBASE_STEPS, its period
                                of exact rebases, so that results do not depend
                                on it */
  int32_t queue_order;       /* order of each round's work queue (counting sort
                                on 15-bit keys): 0 = lowest rigidity E/Z first
                                (the longest histories start first), 1 = by grid
                                brick (neighbouring lanes gather nearby cells),
                                -1 = unsorted.  Results do not depend on it. */
  int32_t use_graph;         /* 1: run the round loop as one captured CUDA graph (a
                                while node; the loop condition is set on the device,
                                so rounds need no host round trip; the graph is kept
                                and replayed while the launch parameters stay the
                                same); 0: host-driven rounds.  Same results. */
  int32_t reserved0;
  const crp_gmf* gmf;        /* with CRP_GMF: the multi-arm field's parameters (host
                                memory, read during the call); else ignored */
} crp_modules;

typedef struct {
  uint64_t accepted_steps;   /* module cycles completed */
  uint64_t rejected_trials;  /* Cash-Karp trials rejected by the controller */
  uint64_t rhs_evals;        /* field gathers + Lorentz evaluations */
  uint64_t n_pion, n_pd;     /* interactions */
  uint64_t n_secondaries;    /* secondaries appended to the pool */
  uint64_t n_dropped;        /* secondaries below e_min, not propagated */
  uint64_t n_overflow;       /* secondaries lost to a full pool */
  uint64_t n_active;         /* candidates still active after the call */
  uint64_t n_detected;       /* candidates detected by the observer (pool total) */
  double kernel_ms;          /* device time of the propagate launches */
  uint32_t launches;         /* kernel launches issued by the call */
  uint32_t error_word;       /* kernel error bits (0 = none) */
} crp_stats;

/* Run the module list on every active candidate in the pool (and on every
 * secondary they spawn) until none is active.  Returns CRP_E_TIMEOUT if the
 * step budget or deadline ran out first (state stays resumable: call again),
 * CRP_E_QUEUE_FULL if secondaries were lost to the pool capacity.  stats_out
 * may be NULL.  Synchronises `stream`. */
crp_status crp_propagate(crp_context* ctx, const crp_grid* grid, const crp_modules* m,
                         void* stream, crp_stats* stats_out);

/* ------------------------------------------------------------------------
 * Output (Sect. 3, output modules: store candidates on detection or at the
 * end).  One record per candidate.
 * ---------------------------------------------------------------------- */
#define CRP_ACTIVE 0
#define CRP_BELOW_EMIN 1
#define CRP_MAX_LENGTH 2
#define CRP_DETECTED 3
#define CRP_AT_BORDER 4
#define CRP_BUDGET 5

typedef struct {
  uint64_t id, parent_id;    /* parent_id 0 for primaries */
  double x[3], u[3];         /* final position, direction */
  double E, s;               /* final energy [eV], trajectory length */
  double x0[3], u0[3];       /* at injection / creation */
  double E0, s_max;
  uint64_t n_acc, n_rej;     /* accepted steps, rejected trials */
  int32_t A, Z, A0, Z0, q;
  int32_t status;            /* CRP_ACTIVE ... CRP_BUDGET */
  uint32_t n_pion, n_pd, draws, generation, n_dropped, lens_pixel;
} crp_record;                /* 208 bytes */

#define CRP_COLLECT_ALL 0
#define CRP_COLLECT_FINISHED 1
#define CRP_COLLECT_DETECTED 2
#define CRP_COLLECT_ACTIVE 3
#define CRP_COLLECT_AT_BORDER 4

/* Copy the records selected by `what`, in pool order, into `out` (host or
 * device memory per out_on_device; capacity records).  *n_out receives the
 * number selected; CRP_E_INVALID if capacity is too small (nothing copied).
 * out = NULL with capacity 0 only counts (size query). */
crp_status crp_collect(crp_context* ctx, int32_t what, crp_record* out, size_t capacity,
                       size_t* n_out, int32_t out_on_device, void* stream);

/* ------------------------------------------------------------------------
 * Galactic lens (Sect. 4, "Galactic propagation": transformation matrices,
 * one per energy bin, map the directions of cosmic rays at the border of
 * the Galaxy to the directions observed at Earth; built by tracking through
 * a galactic field model).
 *
 * Build: antiparticles (charge sign -1, A = Z = 1) leave `earth` along the
 * sample arrival directions dirs[k] with energy E[k] (eV; rigidity E/e) and
 * are propagated with `m` (which must include CRP_BORDER) through `galaxy`
 * in a private pool (the context's own candidates are not touched).  A
 * sample that reaches the border adds its Earth pixel i (HEALPix RING pixel
 * of dirs[k]) to column j (pixel of its direction at the border) of bin
 * bin[k].  Columns keep their samples' Earth pixels sorted ascending.
 * Apply: for each selected candidate with Z > 0, rigidity R = E/Z picks bin
 * b = floor((ln R - ln r_lo) * n_bins / (ln r_hi - ln r_lo)) clamped to the
 * first / last bin, and the arrival direction -u picks column j.  With the
 * uniforms (u1, u2) of Philox draw 0, tag 3 of the candidate's id it is
 * observed if u1 * max_b < count_j (max_b: largest column count of the
 * bin), at Earth pixel entries[min(floor(u2 count_j), count_j - 1)];
 * otherwise lens_pixel = CRP_LENS_NOT_OBSERVED.  Neutral candidates get
 * CRP_LENS_NOT_APPLIED.  The result is in crp_record.lens_pixel.  Every
 * decision (pixel, bin, observed, pick) is that of binary64 arithmetic; the
 * library takes it in binary32 where an error bound shows the two agree and
 * in binary64 otherwise.
 * ---------------------------------------------------------------------- */
#define CRP_LENS_NOT_APPLIED 0xFFFFFFFFu
#define CRP_LENS_NOT_OBSERVED 0xFFFFFFFEu

typedef struct {
  int32_t nside;             /* HEALPix resolution (RING), 1..8192 */
  int32_t n_bins;            /* rigidity bins, log-uniform edges over [r_lo, r_hi] */
  double r_lo, r_hi;         /* rigidity range [V] */
  double earth[3];           /* observer position (length unit of m) */
  const double* dirs;        /* host [n_samples][3] unit arrival directions */
  const double* E;           /* host [n_samples] energies [eV] */
  const int32_t* bin;        /* host [n_samples] rigidity bin of each sample */
  int64_t n_samples;
} crp_lens_desc;

crp_status crp_lens_build(crp_context* ctx, const crp_grid* galaxy, const crp_modules* m,
                          const crp_lens_desc* d, crp_lens** out, crp_stats* stats_out);
crp_status crp_lens_apply(crp_context* ctx, const crp_lens* lens, int32_t what, void* stream);
/* Copy the lens to host memory: col_start (n_bins * 12 nside^2 + 1 entries,
 * columns ordered by bin then border pixel), entries (*n_entries), max_count
 * (n_bins).  Any of the three arrays may be NULL. */
crp_status crp_lens_copy_out(const crp_lens* lens, uint32_t* col_start, uint32_t* entries,
                             uint32_t* max_count, int64_t* n_entries);
crp_status crp_lens_destroy(crp_lens* lens);
/* A lens that takes, for each rigidity bin, the columns of lens b where
 * take_b[bin] != 0 and those of lens a elsewhere (host array of n_bins
 * flags); max_count per bin from the same lens.  Lens normalisation is per
 * bin (Sect. 4 lenses are per rigidity), so a merged bin behaves exactly as
 * in its source lens.  The use: a lens whose bins come from the surrogate
 * where its validated angular error is small enough and from back-tracking
 * elsewhere.  a and b must share device, nside, bins and rigidity range
 * (else CRP_E_INVALID); both stay owned by the caller; synchronous. */
crp_status crp_lens_merge(const crp_lens* a, const crp_lens* b, const uint8_t* take_b,
                          crp_lens** out);

/* ------------------------------------------------------------------------
 * Learned lens surrogate: an MLP that maps an arrival direction at Earth and
 * the log rigidity to the direction at the galaxy border -- a stand-in for
 * back-tracking (Sect. 4: forward and back-tracking through the galactic
 * field) when building lenses.  The paper has no learned component.
 * Inputs (n_x, n_y, n_z, log10(R / V) - 19, ...) FP32 [n][n_in]; n_hidden
 * ReLU layers of width `hidden` (a multiple of 128); a linear 3-output
 * normalised to a unit vector.  Loss mean(1 - y_hat . t).  Hidden-to-hidden
 * layers run on the BF16 tensor cores with FP32 accumulation; master weights,
 * gradients and Adam (beta 0.9 / 0.999, eps 1e-8, bias corrected) in FP32.
 * Parameters packed [W1, b1, ..., W_L+1, b_L+1], W_l (n_out, n_in) row-major.
 * Weights are initialised He-normal from Philox (tag 4, id = index), biases 0.
 * ---------------------------------------------------------------------- */
crp_status crp_mlp_create(crp_context* ctx, int32_t n_in, int32_t hidden, int32_t n_hidden,
                          uint64_t seed, crp_mlp** out);
crp_status crp_mlp_destroy(crp_mlp* mlp);
int64_t crp_mlp_num_params(const crp_mlp* mlp);
/* host FP32 arrays of crp_mlp_num_params entries (resets the Adam state) */
crp_status crp_mlp_set_params(crp_mlp* mlp, const float* params);
/* either pointer may be NULL; grad is the last train step's gradient */
crp_status crp_mlp_get_params(const crp_mlp* mlp, float* params, float* grad);
/* device pointers (either may be NULL when n = 0, which does nothing); n a
 * multiple of 128; y_hat [n][3].  With hidden = 256 and
 * n_in <= 8 the default path is one fused kernel on the fifth-generation
 * tensor cores (tcgen05 MMAs into TMEM, activations kept on chip; it
 * synchronises the stream to read its completion flag and returns CRP_E_CUDA
 * if a tensor-core wait timed out); otherwise, or when selected, one
 * warp-level BF16 GEMM per hidden layer.  Both keep activations in bf16 and
 * accumulate in FP32. */
crp_status crp_mlp_forward(crp_mlp* mlp, const float* x, float* y_hat, int64_t n, void* stream);

#define CRP_MLP_PATH_AUTO 0                /* fused tensor-core kernel when supported */
#define CRP_MLP_PATH_TENSOR_CORE_FUSED 1   /* require it (CRP_E_INVALID if unsupported) */
#define CRP_MLP_PATH_LAYERED 2             /* one GEMM launch per hidden layer */
/* Kernel selection of crp_mlp_forward and crp_mlp_train_step.  With hidden =
 * 256 and n_in <= 8, AUTO / TENSOR_CORE_FUSED train on the fifth-generation
 * tensor cores (tcgen05 GEMMs fed by TMA, FP32 accumulation in TMEM); LAYERED
 * (and every other shape) trains with warp-level mma.sync GEMMs. */
crp_status crp_mlp_set_forward_path(crp_mlp* mlp, int32_t path);
/* one Adam step on a batch (device x [n][n_in], t [n][3] unit targets; n a
 * multiple of 128); lr = 0 computes the gradient only; loss_out (host, may
 * be NULL) receives the batch loss and synchronises the stream (and reports
 * CRP_E_CUDA if a tensor-core wait of this or an earlier step timed out).
 * On the tensor-core path an Adam step is replayed from a CUDA graph after
 * its first call for a batch size (x and t are copied into staging buffers
 * the graph reads); the workspace and staging buffers are shared by the
 * MLP's calls, so steps on different streams must be ordered by the caller. */
crp_status crp_mlp_train_step(crp_mlp* mlp, const float* x, const float* t, int64_t n, float lr,
                              float* loss_out, void* stream);
/* enable != 0 (the default): graph replay of the training step as above;
 * 0: every step launched kernel by kernel (the same arithmetic). */
crp_status crp_mlp_set_train_graph(crp_mlp* mlp, int32_t enable);

/* A lens whose border directions come from the surrogate network instead
 * of back-tracking: sample k's network input is (dirs[k], log10(E[k]/eV) - 19)
 * and its border pixel is the pixel of the predicted direction; the columns
 * are built as in crp_lens_build (d->earth is not used). */
crp_status crp_lens_build_surrogate(crp_context* ctx, crp_mlp* mlp, const crp_lens_desc* d,
                                    crp_lens** out);

/* HEALPix RING arrival map of the selected records: source 0 counts the
 * arrival direction -u at the candidate (extragalactic sky), source 1 the
 * lens_pixel (sky at Earth; shadowed / not applied are skipped).  out: host
 * uint64 array of 12 nside^2 bins. */
crp_status crp_histogram_healpix(crp_context* ctx, int32_t what, int32_t nside, int32_t source,
                                 uint64_t* out, void* stream);

/* The same map counted into the caller's device array out_dev (12 nside^2
 * uint64 on the context's device, 8-byte aligned, else CRP_E_INVALID):
 * cleared first, or added to when accumulate != 0.  Asynchronous on
 * `stream`; no allocation, no synchronisation.  The candidates are
 * independent (Sect. 3), so the map of a job sharded over ranks by
 * candidate is the sum of the ranks' maps: a collective (sum) over these
 * arrays merges them on the devices. */
crp_status crp_histogram_healpix_device(crp_context* ctx, int32_t what, int32_t nside,
                                        int32_t source, uint64_t* out_dev, int32_t accumulate,
                                        void* stream);

/* Histogram over the selected records: nbins log-uniform bins of E over
 * [e_lo, e_hi) (under/overflow dropped).  out: host uint64 array of nbins. */
crp_status crp_histogram_energy(crp_context* ctx, int32_t what, double e_lo, double e_hi,
                                int32_t nbins, uint64_t* out, void* stream);

/* The same histogram counted into the caller's device array out_dev (nbins
 * uint64 on the context's device, 8-byte aligned): cleared first, or added
 * to when accumulate != 0.  Asynchronous on `stream`; no allocation, no
 * synchronisation, so per-rank spectra can be merged on the device by a
 * collective (sum) before anything returns to the host. */
crp_status crp_histogram_energy_device(crp_context* ctx, int32_t what, double e_lo, double e_hi,
                                       int32_t nbins, uint64_t* out_dev, int32_t accumulate,
                                       void* stream);

/* The magnetic field at n points (host arrays xyz [n][3] and B_out [n][3],
 * binary64, the length and field units of the grid) exactly as the
 * propagate kernels of m->precision evaluate it: the grid's trilinear
 * interpolation (Sect. 4: grids for fast lookup) plus, with CRP_GALACTIC in
 * m->flags, the analytic disk and halo field of m, and with CRP_GMF the
 * multi-arm field of m->gmf.  CRP_FP64: binary64 nested
 * interpolation; CRP_MIXED: binary32 (from the cell polynomial records when
 * the grid has them).  Synchronous. */
crp_status crp_grid_sample(const crp_grid* grid, const crp_modules* m, int64_t n,
                           const double* xyz, double* B_out);

/* ---------------------------------------------------------------------
 * 1D mode with cosmology and the a-posteriori 3D cosmology correction.
 * Sect. 2 lists the 1D mode with cosmological effects (redshift evolution
 * of the photon backgrounds, adiabatic expansion); Sect. 4 ("Cosmology in
 * 3D") corrects a 3D run made without cosmology by re-simulating each
 * observed particle in 1D and substituting one of the 1D products.
 * Flat Lambda-CDM.  In 1D a candidate's x holds its redshift; it moves
 * toward the observer in redshift steps (see crp_propagate_1d).
 * ------------------------------------------------------------------- */
typedef struct {
  double H0_km_s_Mpc;  /* 0 = 67.3 */
  double omega_m;      /* 0 = 0.315 (omega_lambda = 1 - omega_m) */
  double dz_max;       /* largest redshift step (0 = 1e-3) */
  double loss_max;     /* largest relative pair loss per step (0 = 1e-3) */
} crp_cosmology;

/* Propagate the context's candidates in 1D: x = source redshift (y, z and
 * the direction are carried but not used).  Uses from m: flags (CRP_PAIR,
 * CRP_ADIABATIC, CRP_PION, CRP_PHOTODIS, CRP_DECAY, CRP_EMIN), e_min,
 * tables (z = 0 rates), length_unit_m, max_steps.  A step lowers z by dz,
 * the smallest of dz_max, the step of relative pair loss loss_max, z, and
 * the step that uses up a stochastic process's remaining optical depth
 * (-ln u at each reset; the event happens at the step's end); its comoving
 * length is dz / H(z - dz/2).  Pair loss with the start-of-step rate, then
 * the exact adiabatic factor (1+z')/(1+z); per comoving length a rate is
 * (1+z)^2 times its table value at (1+z) Gamma (background (1+z)^3 denser,
 * (1+z) hotter); free-neutron decay 1 / ((1+z) gamma c tau).  Arrival at
 * z = 0: CRP_DETECTED.  Records: x = final redshift, x0 = starting redshift,
 * s = comoving length travelled.  Binary64, one candidate per thread. */
crp_status crp_propagate_1d(crp_context* ctx, const crp_cosmology* cosmo, const crp_modules* m,
                            void* stream, crp_stats* stats_out);

/* The a-posteriori correction for n particles observed in a 3D run without
 * cosmology (host arrays): particle i, injected with energy E0[i] and
 * species (A0[i], Z0[i]) and observed after trajectory length T[i] (length
 * units, read as a comoving distance), is re-propagated in 1D from the
 * redshift whose comoving distance is T[i] (seed of ctx, ids id[i]).  Of its
 * products that reach z = 0, ordered by id, product k = min(floor(u n_k),
 * n_k - 1) replaces it (u: Philox counter (0, tag 5, id)); E_out, A_out,
 * Z_out receive it and n_products[i] = n_k (0: nothing arrives; outputs 0).
 * Uses a private pool of n (max A0 + 1) candidates. */
crp_status crp_cosmology_correct(crp_context* ctx, const crp_cosmology* cosmo,
                                 const crp_modules* m, int64_t n, const uint64_t* id,
                                 const double* T, const double* E0, const int32_t* A0,
                                 const int32_t* Z0, double* E_out, int32_t* A_out,
                                 int32_t* Z_out, int32_t* n_products);

/* The pick step of crp_cosmology_correct alone, from given source redshifts
 * (Sect. 4, "Cosmology in 3D"): particle i is re-propagated in 1D from
 * redshift z_src[i] (host array, finite and >= 0, else CRP_E_INVALID) with
 * energy E0[i] and species (A0[i], Z0[i]), and replaced by one of its
 * products that reach z = 0 exactly as crp_cosmology_correct describes.
 * crp_cosmology_correct is crp_redshift_of_distance followed by this call.
 * Host arrays, caller-owned; uses a private pool of n (max A0 + 1)
 * candidates on the context's device and seed. */
crp_status crp_cosmology_pick(crp_context* ctx, const crp_cosmology* cosmo,
                              const crp_modules* m, int64_t n, const uint64_t* id,
                              const double* z_src, const double* E0, const int32_t* A0,
                              const int32_t* Z0, double* E_out, int32_t* A_out,
                              int32_t* Z_out, int32_t* n_products);

/* Redshift at comoving distance D[i] (length units of m) for the cosmology
 * (Gauss-Legendre quadrature of 1 / H; Newton iterations on D(z), kept
 * inside a bracket by bisection). */
crp_status crp_redshift_of_distance(const crp_cosmology* cosmo, double length_unit_m, int64_t n,
                                    const double* D, double* z_out);

/* Launch-configuration autotuner (no counterpart in the paper; the
 * scheduler's tunables are this library's own).  Times crp_propagate on the
 * context's injected candidates under a fixed set of configurations (block
 * size x resident blocks per SM x slice x spatial sort), each started from
 * the same snapshot of the pool and either run to completion
 * (steps_per_trial 0 or UINT64_MAX: the default; it also scores the end of
 * the run, where few candidates are left) or stopped after steps_per_trial
 * accepted steps (steady state only), scored by accepted steps per second of
 * wall time, after one unscored warm-up run.  The pool is restored afterwards:
 * the context is left exactly as it was.  The fastest configuration is
 * written into m (block_size, blocks_per_sm, slice, queue_order) and *out.
 * Results of a propagation do not depend on these settings (every slice
 * tried is a multiple of CRP_MIXED_REBASE_STEPS), so tuning changes speed only.  Needs a
 * device snapshot of the pool (its payload size); CRP_E_INVALID if no
 * candidates are injected. */
typedef struct crp_tune_result {
  int32_t block_size;
  int32_t blocks_per_sm;
  uint32_t slice;
  int32_t queue_order;
  double steps_per_s;  /* of the chosen configuration */
  int32_t n_tried;
  int32_t reserved;
} crp_tune_result;
crp_status crp_autotune(crp_context* ctx, const crp_grid* grid, crp_modules* m,
                        uint64_t steps_per_trial, crp_tune_result* out, void* stream);

/* Checkpoint / restore of a propagation.  Sect. 3 puts the whole state of a
 * particle in its candidate (the stochastic-interaction states included);
 * with per-candidate RNG counters the pool and the seed are therefore the
 * whole state of a propagation, and a restored context continues it
 * bit-identically (for instance after crp_propagate returned CRP_E_TIMEOUT).
 *
 * crp_checkpoint writes a self-describing image of the context into a host
 * buffer: a header (magic, format version, seed, candidate count, element
 * sizes, FNV-1a checksum of the payload) followed by each pool array's first
 * `size` entries.  host_buf = NULL (or capacity 0) is a size query: *n_out
 * receives the bytes needed.  A buffer smaller than that is CRP_E_INVALID.
 * Synchronises `stream`; the caller owns the buffer.
 *
 * crp_restore replaces the context's candidates and seed by the image's.
 * Rejected with CRP_E_INVALID (context unchanged): another format version,
 * a truncated or corrupted image (checksum), or more candidates than the
 * context's capacity.  Synchronises `stream`. */
crp_status crp_checkpoint(crp_context* ctx, void* host_buf, size_t capacity, size_t* n_out,
                          void* stream);
crp_status crp_restore(crp_context* ctx, const void* host_buf, size_t n, void* stream);

/* Measured roofline denominators of a device (no counterpart in the paper):
 * binary32 and binary64 fused multiply-add throughput (2 flops per FMA;
 * each thread runs 8 independent chains over a grid of 8 blocks of 256 per
 * SM) and the read bandwidth of an L2-resident buffer (a quarter of the L2,
 * read 64 times with 16-byte L2-only loads); best of three timed launches
 * after a warm-up.  Allocates and frees one buffer of a quarter of the L2;
 * runs on a private stream and synchronises it. */
typedef struct crp_peaks {
  double fp32_tflops;
  double fp64_tflops;
  double l2_read_gbs;
  int32_t sm_count;
  int32_t l2_bytes;
} crp_peaks;
crp_status crp_measure_peaks(int32_t device, crp_peaks* out);

/* The energy histogram of crp_histogram_energy, counted without allocating
 * anything.  This entry point has no counterpart in the paper: it is for
 * callers that cannot allocate device memory while they run -- their device
 * memory is handed out entirely by another allocator, an allocation failure part way through is not
 * acceptable to them, or they must avoid the device-wide synchronisation
 * that freeing memory can cause.  It calls no cudaMalloc, cudaFree or other
 * allocating routine: the bins are one fixed device array of
 * CRP_HIST_NOALLOC_MAX_BINS 64-bit counters (32 KiB), present on every GPU
 * that loads the library until the process exits.
 *   - nbins above CRP_HIST_NOALLOC_MAX_BINS is rejected with CRP_E_INVALID.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - Every call shares the one array of its device: the call clears the
 *     bins it uses and the array keeps the last call's counts.  Calls in one
 *     process are serialised per device (a lock held from the clearing to
 *     the end of the copy back), so calls from other threads or streams
 *     wait rather than race; each process has its own array.
 *   - Results equal crp_histogram_energy's.  Synchronises `stream`. */
#define CRP_HIST_NOALLOC_MAX_BINS 4096
crp_status crp_histogram_energy_noalloc(crp_context* ctx, int32_t what, double e_lo, double e_hi,
                                        int32_t nbins, uint64_t* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CRP_H_ */
