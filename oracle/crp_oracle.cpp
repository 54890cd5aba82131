// crp_oracle.cpp -- plain, slow, FP64 CPU oracle for the candidate propagation
// method of CRPropa 3.0 (Alves Batista et al., ICRC 2013, arXiv:1307.2643).
//
// TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
// CUDA path is checked against.  Only the test suite, the smoke check and the
// CPU-baseline leg of the benchmark may load it.  It shares no source, header,
// table or constant generator with the GPU library; every formula is written
// out here again from its published source.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared (no FMA
// contraction, so each expression is rounded exactly as written).
//
// What follows the paper directly (Sect. 3, "Cosmic Ray Candidate and
// Modules", and Fig. 1):
//   * the candidate holds its whole propagation state (position, direction,
//     energy, trajectory length, interaction states), so candidates are
//     independent and can be processed concurrently;
//   * the module list is applied in order -- integration (deflection in the
//     field; updates position, direction, trajectory length), interaction
//     modules (continuous losses, stochastic interactions), boundary and
//     observer modules -- and the IsActive flag is checked after each full
//     cycle of the list;
//   * stochastic interaction modules decide independently whether an
//     interaction happens in the current step; after any interaction the
//     states of all interactions are reset;
//   * interactions append secondaries to the candidate's secondary list.
// The paper prints no equations.  Every formula below therefore comes from
// the textbook or published method named beside it; where the paper is silent
// the chosen reading is stated in a comment marked "reading".

#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>
#include <atomic>

namespace {

// ---------------------------------------------------------------------------
// Physical constants: CODATA 2018 exact / recommended values, IAU parsec.
// ---------------------------------------------------------------------------
const double kC = 299792458.0;                  // speed of light [m/s]
const double kMeC2 = 0.51099895000e6;           // electron rest energy [eV]
const double kMpC2 = 938.27208816e6;            // proton rest energy [eV]
const double kMnC2 = 939.56542052e6;            // neutron rest energy [eV] (CODATA 2018)
const double kTauN = 878.4;                     // free-neutron mean lifetime [s] (reading)
const double kAlpha = 7.2973525693e-3;          // fine-structure constant
const double kRe = 2.8179403262e-15;            // classical electron radius [m]
const double kKB = 8.617333262e-5;              // Boltzmann constant [eV/K]
const double kHbarC = 1.973269804e-7;           // hbar*c [eV m]
const double kPi = 3.14159265358979323846;
const double kMillibarn = 1.0e-31;              // [m^2]

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator, written from its definition in
// J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11 (2011): ten rounds of two 32x32->64
// multiplications (multipliers 0xD2511F53 and 0xCD9E8D57) with a Weyl key
// schedule (increments 0x9E3779B9 and 0xBB67AE85).
// ---------------------------------------------------------------------------
struct Words4 { uint32_t w[4]; };

Words4 philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {                      // key bump between rounds
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  Words4 r;
  r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
  return r;
}

// Two 32-bit words -> a double in the open interval (0, 1): the top 52 bits
// of the 64-bit word (w_hi:w_lo), offset by one half, times 2^-52.  Every
// value is exact in binary64 (reading: the paper does not fix the RNG).
double uniform_open(uint32_t w_lo, uint32_t w_hi) {
  uint64_t v = ((uint64_t)w_hi << 32) | (uint64_t)w_lo;
  return ((double)(v >> 12) + 0.5) * (1.0 / 4503599627370496.0);
}

// Stream tags of the counter layout (draw index, tag, id_lo, id_hi).
const uint32_t kTagField = 1;
const uint32_t kTagInteraction = 2;

Words4 draw_words(uint64_t seed, uint32_t tag, uint64_t id, uint32_t draw_idx) {
  uint32_t ctr[4] = {draw_idx, tag, (uint32_t)id, (uint32_t)(id >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  return philox4x32_10(ctr, key);
}

// SplitMix64 output function (G. L. Steele, D. Lea, C. H. Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014): the finaliser
// that turns a Weyl-sequence state into a well-mixed 64-bit value.
uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Lineage-derived id of the secondary emitted in the parent's event number
// `event_index` (reading: ids must not depend on processing order).
uint64_t child_id(uint64_t parent_id, uint32_t event_index) {
  return splitmix64_mix(parent_id + 0x9E3779B97F4A7C15ULL * ((uint64_t)event_index + 1ULL));
}

// ---------------------------------------------------------------------------
// Natural logarithm by the classical atanh series (reading: both the oracle
// and the GPU library evaluate the logarithms that steer the propagation --
// interaction free paths -ln(u) and the ln(Gamma) of table lookups -- with
// this one formula, so that those values agree bit for bit; a library log
// may differ by an ulp, and the adaptive step controller turns an ulp into a
// different step sequence).
//   x = 2^k m with m in [sqrt(1/2), sqrt(2)],  s = (m - 1)/(m + 1),
//   ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + ... + s^26/27),
//   ln x = k ln 2 + ln m.
// Valid for positive normal finite x; |s| <= 0.172, so the truncated tail is
// below 1e-21 and the result is within a few ulp of ln x.
// ---------------------------------------------------------------------------
double series_log(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  int k = (int)((b >> 52) & 0x7ff) - 1023;
  uint64_t mb = (b & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL;
  double m;
  std::memcpy(&m, &mb, sizeof(m));
  if (m > 1.4142135623730951) {
    m = m * 0.5;
    k = k + 1;
  }
  const double s = (m - 1.0) / (m + 1.0);
  const double z = s * s;
  double poly = 1.0 / 27.0;
  poly = poly * z + 1.0 / 25.0;
  poly = poly * z + 1.0 / 23.0;
  poly = poly * z + 1.0 / 21.0;
  poly = poly * z + 1.0 / 19.0;
  poly = poly * z + 1.0 / 17.0;
  poly = poly * z + 1.0 / 15.0;
  poly = poly * z + 1.0 / 13.0;
  poly = poly * z + 1.0 / 11.0;
  poly = poly * z + 1.0 / 9.0;
  poly = poly * z + 1.0 / 7.0;
  poly = poly * z + 1.0 / 5.0;
  poly = poly * z + 1.0 / 3.0;
  poly = poly * z + 1.0;
  const double ln_m = 2.0 * s * poly;
  return (double)k * 0.69314718055994530942 + ln_m;
}

// Exponential for the analytic galactic field, written out so that an
// independent binary64 implementation reproduces it bit for bit (reading:
// as for the logarithm, a library exp may differ by an ulp).  Range
// reduction x = k ln2 + r with k = nearest integer of x/ln2, ln2 split in a
// 32-bit high part (k * high is exact) and a low part (Cody & Waite),
// |r| <= ln2/2; e^r by its
// Taylor series to r^13/13! (Horner; tail below 1e-17); 2^k applied by
// building the exponent field.  Valid for -700 <= x <= 700.
double series_exp(double x) {
  if (x < -700.0) return 0.0;
  const double ln2_hi = 2977044472.0 / 4294967296.0;  // ln 2 to 32 bits (exact)
  const double ln2_lo = -4.2009150726810847e-11;       // ln 2 - ln2_hi
  double kd = std::floor(x * 1.4426950408889634074 + 0.5);
  double r = (x - kd * ln2_hi) - kd * ln2_lo;
  double poly = 1.0 / 6227020800.0;                 // 1/13!
  poly = poly * r + 1.0 / 479001600.0;              // 1/12!
  poly = poly * r + 1.0 / 39916800.0;
  poly = poly * r + 1.0 / 3628800.0;
  poly = poly * r + 1.0 / 362880.0;
  poly = poly * r + 1.0 / 40320.0;
  poly = poly * r + 1.0 / 5040.0;
  poly = poly * r + 1.0 / 720.0;
  poly = poly * r + 1.0 / 120.0;
  poly = poly * r + 1.0 / 24.0;
  poly = poly * r + 1.0 / 6.0;
  poly = poly * r + 1.0 / 2.0;
  poly = poly * r + 1.0;
  poly = poly * r + 1.0;
  int k = (int)kd;
  uint64_t bits = (uint64_t)(k + 1023) << 52;
  double scale;
  std::memcpy(&scale, &bits, sizeof(scale));
  return poly * scale;
}

// Arctangent of y/x in (-pi, pi], by argument halving and the Taylor series of
// atan (reading: the spiral phase of the multi-arm galactic field is steered by
// this one formula on both sides, for the reason given at series_log).
//   t = min(|x|,|y|) / max(|x|,|y|) in [0, 1];
//   three halvings atan t = 2 atan(t / (1 + sqrt(1 + t^2))) bring t below
//   tan(pi/32) < 0.0985, where atan t = t - t^3/3 + t^5/5 - ... - t^15/15
//   leaves a tail below 1e-17 t;
//   then atan(1/t) = pi/2 - atan t, atan2(y, -x) = pi - atan2(y, x) and
//   atan2(-y, x) = -atan2(y, x).  atan2(0, 0) = 0.
double series_atan2(double y, double x) {
  const double ax = std::fabs(x), ay = std::fabs(y);
  if (ax == 0.0 && ay == 0.0) return 0.0;
  const bool steep = ay > ax;
  double t = steep ? ax / ay : ay / ax;
  for (int i = 0; i < 3; ++i) t = t / (1.0 + std::sqrt(1.0 + t * t));
  const double t2 = t * t;
  double poly = -1.0 / 15.0;
  poly = poly * t2 + 1.0 / 13.0;
  poly = poly * t2 - 1.0 / 11.0;
  poly = poly * t2 + 1.0 / 9.0;
  poly = poly * t2 - 1.0 / 7.0;
  poly = poly * t2 + 1.0 / 5.0;
  poly = poly * t2 - 1.0 / 3.0;
  poly = poly * t2 + 1.0;
  double a = 8.0 * (t * poly);
  if (steep) a = 0.5 * kPi - a;
  if (x < 0.0) a = kPi - a;
  return y < 0.0 ? -a : a;
}

// ---------------------------------------------------------------------------
// HEALPix RING scheme (K. M. Gorski et al., "HEALPix: a framework for high
// resolution discretization and fast analysis of data distributed on the
// sphere", ApJ 622, 759 (2005)): 12 nside^2 equal-area pixels; rings of
// constant z = cos(theta); polar caps |z| > 2/3 and the equatorial belt.
// Pixel index of a unit direction, and the centre of a pixel.
// ---------------------------------------------------------------------------
int64_t healpix_ang2pix_ring(int64_t nside, double z, double phi) {
  const double pi = kPi;
  const double twopi = 2.0 * kPi;
  phi = std::fmod(phi, twopi);
  if (phi < 0.0) phi += twopi;
  const double tt = phi / (0.5 * pi);               // in [0, 4)
  const double za = std::fabs(z);
  const int64_t ncap = 2 * nside * (nside - 1);
  const int64_t npix = 12 * nside * nside;
  if (za <= 2.0 / 3.0) {                           // equatorial belt
    const double t1 = (double)nside * (0.5 + tt);
    const double t2 = (double)nside * z * 0.75;
    const int64_t jp = (int64_t)std::floor(t1 - t2);  // ascending edge line
    const int64_t jm = (int64_t)std::floor(t1 + t2);  // descending edge line
    const int64_t ir = nside + 1 + jp - jm;            // ring index from z = 2/3, 1..2nside+1
    const int64_t kshift = 1 - (ir & 1);
    int64_t ip = (jp + jm - nside + kshift + 1) / 2;
    ip = ((ip % (4 * nside)) + 4 * nside) % (4 * nside);
    return ncap + (ir - 1) * 4 * nside + ip;
  }
  const double tp = tt - std::floor(tt);
  const double tmp = (double)nside * std::sqrt(3.0 * (1.0 - za));
  const int64_t jp = (int64_t)std::floor(tp * tmp);
  const int64_t jm = (int64_t)std::floor((1.0 - tp) * tmp);
  const int64_t ir = jp + jm + 1;                  // ring index from the pole
  int64_t ip = (int64_t)std::floor(tt * (double)ir);
  ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
  if (z > 0.0) return 2 * ir * (ir - 1) + ip;
  return npix - 2 * ir * (ir + 1) + ip;
}

void healpix_pix2ang_ring(int64_t nside, int64_t pix, double* z, double* phi) {
  const double pi = kPi;
  const int64_t ncap = 2 * nside * (nside - 1);
  const int64_t npix = 12 * nside * nside;
  const double fact2 = 4.0 / (double)npix;
  if (pix < ncap) {                                 // north polar cap
    const int64_t iring = (int64_t)((1.0 + std::sqrt(1.0 + 2.0 * (double)pix)) * 0.5);
    const int64_t iphi = pix + 1 - 2 * iring * (iring - 1);
    *z = 1.0 - (double)(iring * iring) * fact2;
    *phi = ((double)iphi - 0.5) * pi / (2.0 * (double)iring);
  } else if (pix < npix - ncap) {                   // equatorial belt
    const int64_t ip = pix - ncap;
    const int64_t iring = ip / (4 * nside) + nside; // counted from the north pole
    const int64_t iphi = ip % (4 * nside) + 1;
    const double fodd = ((iring + nside) & 1) ? 1.0 : 0.5;
    *z = (double)(2 * nside - iring) * 2.0 / (3.0 * (double)nside);
    *phi = ((double)iphi - fodd) * pi / (2.0 * (double)nside);
  } else {                                          // south polar cap
    const int64_t ip = npix - pix;
    const int64_t iring = (int64_t)((1.0 + std::sqrt(2.0 * (double)ip - 1.0)) * 0.5);
    const int64_t iphi = 4 * iring + 1 - (ip - 2 * iring * (iring - 1));
    *z = -1.0 + (double)(iring * iring) * fact2;
    *phi = ((double)iphi - 0.5) * pi / (2.0 * (double)iring);
  }
}

// ---------------------------------------------------------------------------
// Photon field: Planck spectrum of the CMB.
// n(eps) = eps^2 / (pi^2 (hbar c)^3 (exp(eps/kT) - 1))   [1 / (m^3 eV)]
// ---------------------------------------------------------------------------
double planck_density(double eps, double kT) {
  double x = eps / kT;
  if (x > 700.0) return 0.0;
  return eps * eps / (kPi * kPi * kHbarC * kHbarC * kHbarC * std::expm1(x));
}

// ---------------------------------------------------------------------------
// Bethe-Heitler pair production energy-loss function phi(kappa) of
// G. R. Blumenthal, Phys. Rev. D 1, 1596 (1970), in the analytic
// approximation of M. J. Chodorowski, A. A. Zdziarski, M. Sikora,
// ApJ 400, 181 (1992): a rational form with leading term (pi/12)(k-2)^4
// below kappa = 25, and kappa * cubic-in-ln(kappa) over a rational
// correction above.  kappa is the photon energy in the nucleus rest frame in
// units of m_e c^2; the threshold is kappa = 2.
// ---------------------------------------------------------------------------
double phi_pair(double k) {
  if (k <= 2.0) return 0.0;
  if (k < 25.0) {
    double d = k - 2.0;
    double den = 1.0 + 0.8048 * d + 0.1459 * d * d + 1.137e-3 * d * d * d
                 - 3.879e-6 * d * d * d * d;
    return kPi / 12.0 * d * d * d * d / den;
  }
  double L = std::log(k);
  double num = -86.07 + 50.96 * L - 14.45 * L * L + (8.0 / 3.0) * L * L * L;
  double den = 1.0 - (2.910 / k + 78.35 / (k * k) + 1837.0 / (k * k * k));
  return k * num / den;
}

// Gauss-Legendre rule with n nodes on [-1, 1]: nodes are the roots of the
// Legendre polynomial P_n, found by Newton iteration on the three-term
// recurrence; weights 2 / ((1 - x^2) P_n'(x)^2) (textbook construction).
struct GaussRule {
  std::vector<double> x, w;
};

GaussRule gauss_legendre(int n) {
  GaussRule g;
  g.x.resize(n);
  g.w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    g.x[i] = z;
    g.w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return g;
}

const GaussRule& rule(int n) {
  static const GaussRule g10 = gauss_legendre(10);
  static const GaussRule g20 = gauss_legendre(20);
  return n == 10 ? g10 : g20;
}

template <class F>
double gauss_apply(const F& f, double a, double b, const GaussRule& g) {
  double mid = 0.5 * (a + b), half = 0.5 * (b - a), sum = 0.0;
  for (size_t i = 0; i < g.x.size(); ++i) sum += g.w[i] * f(mid + half * g.x[i]);
  return sum * half;
}

// Adaptive bisection: accept the 20-point value on an interval when it agrees
// with the 10-point value to the absolute tolerance, else split.
template <class F>
double gauss_rec(const F& f, double a, double b, double tol, int depth) {
  double i20 = gauss_apply(f, a, b, rule(20));
  double i10 = gauss_apply(f, a, b, rule(10));
  if (depth <= 0 || std::fabs(i20 - i10) <= tol) return i20;
  if (b - a <= 1e-12 * (std::fabs(a) + std::fabs(b))) return i20;   // rounding floor
  double m = 0.5 * (a + b);
  return gauss_rec(f, a, m, 0.5 * tol, depth - 1) + gauss_rec(f, m, b, 0.5 * tol, depth - 1);
}

// Integral over [a, b] to a relative tolerance of the integral's magnitude,
// starting from 16 equal panels.
template <class F>
double adaptive_quad(const F& f, double a, double b, double rel_tol) {
  if (!(b > a)) return 0.0;
  const int panels = 16;
  double scale = 0.0;
  for (int p = 0; p < panels; ++p)
    scale += std::fabs(gauss_apply(f, a + (b - a) * p / panels, a + (b - a) * (p + 1) / panels,
                                   rule(20)));
  // An integrand that underflows everywhere contributes nothing measurable.
  if (!(rel_tol * scale > 1e-290)) return scale;
  double total = 0.0;
  for (int p = 0; p < panels; ++p)
    total += gauss_rec(f, a + (b - a) * p / panels, a + (b - a) * (p + 1) / panels,
                       rel_tol * scale / panels, 40);
  return total;
}

// Relative energy-loss rate of a proton by pair production on the CMB,
// beta = (1/E) dE/dx [1/m], from Blumenthal (1970):
//   -dE/dt = alpha r_e^2 (m_e c^2)^2 c  int_2^inf dk n(k m_e c^2 / (2 Gamma)) phi(k) / k^2
// with E = Gamma m_p c^2 and dx = c dt.  Integrated over ln(kappa), split at
// kappa = 25 where the two branches of phi meet.
double beta_pair_proton(double gamma, double kT) {
  double kmax = 1400.0 * gamma * kT / kMeC2;   // eps/kT = 700 cut
  if (kmax <= 2.0) return 0.0;
  auto integrand = [&](double y) {
    double k = std::exp(y);
    double eps = k * kMeC2 / (2.0 * gamma);
    return k * planck_density(eps, kT) * phi_pair(k) / (k * k);
  };
  double y2 = std::log(2.0), y25 = std::log(25.0), ym = std::log(kmax);
  double I = 0.0;
  if (ym <= y25) {
    I = adaptive_quad(integrand, y2, ym, 1e-12);
  } else {
    I = adaptive_quad(integrand, y2, y25, 1e-12) + adaptive_quad(integrand, y25, ym, 1e-12);
  }
  double dEdx = kAlpha * kRe * kRe * kMeC2 * kMeC2 * I;   // [eV/m]
  return dEdx / (gamma * kMpC2);
}

// Photo-pion interaction rate of a nucleon [1/m] for a step cross section
// sigma(eps') = sigma0 for eps' > eps_th (rest-frame photon energy).
// The rate on an isotropic photon gas,
//   R = 1/(2 Gamma^2) int d eps n(eps)/eps^2 int_{eps_th}^{2 Gamma eps} eps' sigma(eps') d eps',
// reduces for the step and a Planck n to a Bose-Einstein series in
// x0 = eps_th / (2 Gamma kT):
//   R = 2 sigma0 (kT/hbar c)^3 / pi^2 * sum_n exp(-n x0) (x0/n^2 + 1/n^3).
double rate_pion_nucleon(double gamma, double kT, double sigma0, double eps_th) {
  double x0 = eps_th / (2.0 * gamma * kT);
  double sum = 0.0;
  for (int n = 1; n < 1000000; ++n) {
    double e = std::exp(-n * x0);
    if (e == 0.0) break;
    double term = e * (x0 / ((double)n * n) + 1.0 / ((double)n * n * n));
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  double t = kT / kHbarC;
  return 2.0 * sigma0 * t * t * t / (kPi * kPi) * sum;
}

// Giant-dipole photodisintegration rate per nucleon [1/m].  Synthetic
// Lorentzian cross section (reading of "peak 20 MeV, width 6 MeV, amplitude
// proportional to A"): sigma(eps') = s_pk w^2 / ((eps' - e_c)^2 + w^2) with
// w = FWHM/2, restricted to eps' in [e_lo, e_hi]; the upper cut is needed
// because int eps' sigma d eps' grows logarithmically.  The inner integral
// has the closed form
//   int eps' sigma = s_pk w^2 [ 1/2 ln((eps'-e_c)^2 + w^2) + (e_c/w) atan((eps'-e_c)/w) ];
// the outer integral over the Planck spectrum is done by quadrature in ln eps.
double gdr_inner(double ep, double s_pk, double e_c, double w, double e_lo, double e_hi) {
  if (ep <= e_lo) return 0.0;
  if (ep > e_hi) ep = e_hi;
  // F(ep) - F(e_lo) written without cancellation near the threshold:
  //   ln-part:   1/2 ln(1 + D (d1 + d0) / (d0^2 + w^2))
  //   atan-part: atan(d1/w) - atan(d0/w) = atan2(w D, w^2 + d1 d0)
  // with D = ep - e_lo, d1 = ep - e_c, d0 = e_lo - e_c.
  double D = ep - e_lo, d1 = ep - e_c, d0 = e_lo - e_c;
  double lnpart = 0.5 * std::log1p(D * (d1 + d0) / (d0 * d0 + w * w));
  double atpart = (e_c / w) * std::atan2(w * D, w * w + d1 * d0);
  return s_pk * w * w * (lnpart + atpart);
}

double rate_gdr_nucleon(double gamma, double kT, double s_pk, double e_c, double w,
                        double e_lo, double e_hi) {
  double eps_lo = e_lo / (2.0 * gamma);
  double eps_hi = 700.0 * kT;
  if (eps_hi <= eps_lo) return 0.0;
  auto integrand = [&](double y) {
    double eps = std::exp(y);
    return eps * planck_density(eps, kT) / (eps * eps) *
           gdr_inner(2.0 * gamma * eps, s_pk, e_c, w, e_lo, e_hi);
  };
  double ya = std::log(eps_lo), yb = std::log(eps_hi);
  double ysat = std::log(e_hi / (2.0 * gamma));   // inner integral saturates here
  double I;
  if (ysat > ya && ysat < yb)
    I = adaptive_quad(integrand, ya, ysat, 1e-12) + adaptive_quad(integrand, ysat, yb, 1e-12);
  else
    I = adaptive_quad(integrand, ya, yb, 1e-12);
  return I / (2.0 * gamma * gamma);
}

// ---------------------------------------------------------------------------
// Cash-Karp embedded Runge-Kutta 5(4) tableau: J. R. Cash, A. H. Karp,
// "A variable order Runge-Kutta method for initial value problems with
// rapidly varying right-hand sides", ACM TOMS 16, 201 (1990).  Each constant
// is the nearest double of the published rational.
// ---------------------------------------------------------------------------
const double b21 = 1.0 / 5.0;
const double b31 = 3.0 / 40.0, b32 = 9.0 / 40.0;
const double b41 = 3.0 / 10.0, b42 = -9.0 / 10.0, b43 = 6.0 / 5.0;
const double b51 = -11.0 / 54.0, b52 = 5.0 / 2.0, b53 = -70.0 / 27.0, b54 = 35.0 / 27.0;
const double b61 = 1631.0 / 55296.0, b62 = 175.0 / 512.0, b63 = 575.0 / 13824.0,
             b64 = 44275.0 / 110592.0, b65 = 253.0 / 4096.0;
// fifth-order weights
const double c1 = 37.0 / 378.0, c3 = 250.0 / 621.0, c4 = 125.0 / 594.0, c6 = 512.0 / 1771.0;
// fifth minus embedded fourth order, c_i - c*_i with the fourth-order weights
// c* = (2825/27648, 0, 18575/48384, 13525/55296, 277/14336, 1/4), each
// written as its exact reduced rational so the double is the nearest one
const double e1 = -277.0 / 64512.0;
const double e3 = 6925.0 / 370944.0;
const double e4 = -6925.0 / 202752.0;
const double e5 = -277.0 / 14336.0;
const double e6 = 277.0 / 7084.0;

}  // namespace

// ===========================================================================
// C interface (loaded by ctypes from the test suite).
// ===========================================================================
extern "C" {

// Status of a finished candidate (reading: the paper's IsActive flag,
// refined by which module switched it off).
enum {
  ORC_ACTIVE = 0,
  ORC_BELOW_EMIN = 1,
  ORC_MAX_LENGTH = 2,
  ORC_DETECTED = 3,
  ORC_AT_BORDER = 4,
  ORC_BUDGET = 5,
};

// Module flags.
enum {
  ORC_PAIR = 1u << 0,
  ORC_ADIABATIC = 1u << 1,
  ORC_PION = 1u << 2,
  ORC_PHOTODIS = 1u << 3,
  ORC_EMIN = 1u << 4,
  ORC_OBSERVER = 1u << 5,
  ORC_BORDER = 1u << 6,
  ORC_GALACTIC = 1u << 7,   // add the analytic galactic disk + halo field
  ORC_DECAY = 1u << 8,      // free-neutron beta decay
  ORC_GMF = 1u << 9,        // add the analytic multi-arm galactic field
};

// Parameters of the analytic multi-arm galactic field (units of the field
// grid); the model is stated at gmf_field.
struct orc_gmf {
  double arm_b[8];      // arm field strengths at r = r_in
  double arm_rx[8];     // radii where the arm boundaries cross phi = pi, ascending
  double pitch_rad;     // spiral pitch angle p
  double ring_b;        // azimuthal field of the ring r_ring <= r < r_in
  double r_ring, r_in, r_out;
  double h_disk, w_disk;                       // disk / halo transition
  double halo_bn, halo_bs, halo_rn, halo_rs, halo_wh, halo_z0;
  double x_b, x_theta_rad, x_rc, x_r;          // X-shaped poloidal field
  double r_cut_in, r_cut_out;                  // spherical cuts (0: none)
};

struct orc_params {
  // field grid: node (i,j,k) sits at origin + (i,j,k) * spacing, periodic
  double origin[3];
  double spacing;
  int64_t n[3];
  // integrator
  double tol, h_min, h_max;
  double curv_k;       // c * field unit [T] * length unit [m]  (eV per field*length unit)
  // losses and interactions
  double beta_ad;      // adiabatic loss rate H0/c [1/length]
  double e_min;        // [eV]
  uint32_t flags;
  uint32_t pad0;
  uint64_t seed;
  // rate tables: node i at ln(Gamma) = lg0 + i / inv_dlg
  double tab_lg0, tab_inv_dlg;
  int64_t tab_n;
  // observer sphere and galactic border sphere
  double obs_c[3], obs_r;
  double border_c[3], border_r;
  // analytic galactic field (units of the field grid)
  double gal_disk_b, gal_disk_pitch_rad, gal_disk_hz, gal_disk_rmin, gal_disk_rmax;
  double gal_halo_b, gal_halo_z0, gal_halo_sigma;
  double gal_center[3];
  int64_t max_steps;   // per-candidate accepted-step budget
  double length_unit_m;  // metres per length unit (neutron decay length)
  orc_gmf gmf;           // analytic multi-arm galactic field (ORC_GMF)
  // unstable nuclei (ORC_DECAY; NULL: only free neutrons decay): for
  // 0 <= Z <= A <= nuc_amax, the 5 doubles at nuc_tab + 5 (A (A+1) / 2 + Z)
  // are the rest-frame mean lifetime [s] (infinite: stable) and the
  // branching fractions of beta-, beta+, neutron emission, proton emission
  const double* nuc_tab;
  int64_t nuc_amax;
};

struct orc_record {
  uint64_t id, parent_id;
  double x[3], u[3];
  double E, s;
  double x0[3], u0[3];
  double E0, s_max;
  uint64_t n_acc, n_rej;
  int32_t A, Z, A0, Z0, q;
  int32_t status;
  uint32_t n_pion, n_pd, draws, generation, n_dropped, pad;
};

// -- exported primitives (used by the pins in the test suite) --------------
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  Words4 r = philox4x32_10(ctr, key);
  for (int i = 0; i < 4; ++i) out[i] = r.w[i];
}
double orc_uniform_open(uint32_t lo, uint32_t hi) { return uniform_open(lo, hi); }
// Two uniforms (words 0,1 and 2,3) of draw `draw` with `tag` for each id.
void orc_uniform_pairs(uint64_t seed, uint32_t tag, uint32_t draw, int64_t n, const uint64_t* ids,
                       double* out) {
  for (int64_t i = 0; i < n; ++i) {
    Words4 w = draw_words(seed, tag, ids[i], draw);
    out[2 * i] = uniform_open(w.w[0], w.w[1]);
    out[2 * i + 1] = uniform_open(w.w[2], w.w[3]);
  }
}
uint64_t orc_child_id(uint64_t parent, uint32_t ev) { return child_id(parent, ev); }
double orc_phi_pair(double k) { return phi_pair(k); }
double orc_series_log(double x) { return series_log(x); }
void orc_series_log_vec(int64_t n, const double* x, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = series_log(x[i]);
}
double orc_series_exp(double x) { return series_exp(x); }
void orc_series_atan2_vec(int64_t n, const double* y, const double* x, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = series_atan2(y[i], x[i]);
}
int64_t orc_ang2pix(int64_t nside, double z, double phi) { return healpix_ang2pix_ring(nside, z, phi); }
void orc_pix2ang(int64_t nside, int64_t pix, double* z, double* phi) {
  healpix_pix2ang_ring(nside, pix, z, phi);
}
// Vectorised forms for the lens oracle.
void orc_ang2pix_vec(int64_t nside, int64_t n, const double* u, int64_t* out) {
  for (int64_t i = 0; i < n; ++i) {
    const double x = u[3 * i], y = u[3 * i + 1], z = u[3 * i + 2];
    out[i] = healpix_ang2pix_ring(nside, z, std::atan2(y, x));
  }
}
double orc_planck_density(double eps, double kT) { return planck_density(eps, kT); }
double orc_beta_pair_proton(double gamma, double T) { return beta_pair_proton(gamma, kKB * T); }
double orc_rate_pion_nucleon(double gamma, double T, double sigma0_mb, double eps_th_eV) {
  return rate_pion_nucleon(gamma, kKB * T, sigma0_mb * kMillibarn, eps_th_eV);
}
double orc_rate_gdr_nucleon(double gamma, double T, double s_pk_mb, double e_c, double fwhm,
                            double e_lo, double e_hi) {
  return rate_gdr_nucleon(gamma, kKB * T, s_pk_mb * kMillibarn, e_c, 0.5 * fwhm, e_lo, e_hi);
}
void orc_cash_karp_tableau(double* out) {
  const double v[] = {b21, b31, b32, b41, b42, b43, b51, b52, b53, b54,
                      b61, b62, b63, b64, b65, c1, c3, c4, c6, e1, e3, e4, e5, e6};
  for (int i = 0; i < 24; ++i) out[i] = v[i];
}

// Rate tables on n nodes uniform in ln(Gamma) over [ln g_lo, ln g_hi], in
// units of 1/length_unit_m.  Pair: Blumenthal beta for a proton on the CMB
// plus, for a synthetic infrared / optical background of n_irb dilute
// blackbodies (temperature irb_T[k], dilution irb_D[k]), sum_k D_k times the
// blackbody beta at T_k (the loss rate is linear in the photon density).
// Pion: nucleon rate for the step cross section.  GDR: per-nucleon rate.
void orc_tables_build(int64_t n, double g_lo, double g_hi, double length_unit_m, double T_cmb,
                      double pion_sigma_mb, double pion_eth_eV,
                      double gdr_peak_mb, double gdr_ec_eV, double gdr_fwhm_eV,
                      double gdr_lo_eV, double gdr_hi_eV,
                      double* beta_pair, double* rate_pion, double* rate_gdr, int nthreads,
                      int n_irb, const double* irb_T, const double* irb_D) {
  double kT = kKB * T_cmb;
  double lg0 = std::log(g_lo), lg1 = std::log(g_hi);
  auto work = [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      double gamma = std::exp(lg0 + (lg1 - lg0) * (double)i / (double)(n - 1));
      double b = beta_pair_proton(gamma, kT);
      for (int k = 0; k < n_irb; ++k)
        if (irb_D[k] > 0.0) b = b + irb_D[k] * beta_pair_proton(gamma, kKB * irb_T[k]);
      beta_pair[i] = b * length_unit_m;
      rate_pion[i] = rate_pion_nucleon(gamma, kT, pion_sigma_mb * kMillibarn, pion_eth_eV) * length_unit_m;
      rate_gdr[i] = rate_gdr_nucleon(gamma, kT, gdr_peak_mb * kMillibarn, gdr_ec_eV, 0.5 * gdr_fwhm_eV,
                                     gdr_lo_eV, gdr_hi_eV) * length_unit_m;
    }
  };
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t a = t * chunk, b = std::min<int64_t>(n, a + chunk);
    if (a < b) th.emplace_back(work, a, b);
  }
  for (auto& t : th) t.join();
}

// Turbulent-field Fourier modes.  For every FFT wavevector
// k = 2 pi m / (N spacing) (m in numpy's fftfreq order) with
// 2 pi / lmax <= |k| <= 2 pi / lmin, three complex Gaussian components are
// drawn (Box-Muller on two Philox uniforms per component, tag 1, id = the
// mode's linear index), projected perpendicular to k so that k . B = 0, and
// scaled by |k|^(index/2) so that |B(k)|^2 ~ |k|^index (index = -11/3 for
// Kolmogorov); modes on a Nyquist plane stay zero.  Output: complex modes [nz][ny][nx][3] as (re, im) pairs; the
// field is the real part of their inverse FFT, normalised afterwards.
void orc_turbulence_modes(int64_t nx, int64_t ny, int64_t nz, double spacing, double lmin,
                          double lmax, double index, uint64_t seed, double* out) {
  const double kmin = 2.0 * kPi / lmax, kmax = 2.0 * kPi / lmin;
  for (int64_t iz = 0; iz < nz; ++iz)
    for (int64_t iy = 0; iy < ny; ++iy)
      for (int64_t ix = 0; ix < nx; ++ix) {
        int64_t lin = (iz * ny + iy) * nx + ix;
        double* o = out + lin * 6;
        for (int c = 0; c < 6; ++c) o[c] = 0.0;
        int64_t mx = ix < (nx + 1) / 2 ? ix : ix - nx;
        int64_t my = iy < (ny + 1) / 2 ? iy : iy - ny;
        int64_t mz = iz < (nz + 1) / 2 ? iz : iz - nz;
        double kx = 2.0 * kPi * (double)mx / ((double)nx * spacing);
        double ky = 2.0 * kPi * (double)my / ((double)ny * spacing);
        double kz = 2.0 * kPi * (double)mz / ((double)nz * spacing);
        double k = std::sqrt(kx * kx + ky * ky + kz * kz);
        if (!(k >= kmin && k <= kmax)) continue;
        // Nyquist planes are left empty (reading): there -k aliases onto a
        // mode whose wavevector is not -k, so the real part of the field
        // would not stay divergence free.
        if ((nx % 2 == 0 && 2 * ix == nx) || (ny % 2 == 0 && 2 * iy == ny) ||
            (nz % 2 == 0 && 2 * iz == nz))
          continue;
        double re[3], im[3];
        for (int c = 0; c < 3; ++c) {
          Words4 w = draw_words(seed, kTagField, (uint64_t)lin, (uint32_t)c);
          double u1 = uniform_open(w.w[0], w.w[1]);
          double u2 = uniform_open(w.w[2], w.w[3]);
          double r = std::sqrt(-2.0 * std::log(u1));
          re[c] = r * std::cos(2.0 * kPi * u2);
          im[c] = r * std::sin(2.0 * kPi * u2);
        }
        double hx = kx / k, hy = ky / k, hz = kz / k;
        double pr = hx * re[0] + hy * re[1] + hz * re[2];
        double pi_ = hx * im[0] + hy * im[1] + hz * im[2];
        re[0] -= pr * hx; re[1] -= pr * hy; re[2] -= pr * hz;
        im[0] -= pi_ * hx; im[1] -= pi_ * hy; im[2] -= pi_ * hz;
        double amp = std::pow(k, 0.5 * index);
        for (int c = 0; c < 3; ++c) {
          o[2 * c] = re[c] * amp;
          o[2 * c + 1] = im[c] * amp;
        }
      }
}

}  // extern "C"

// ===========================================================================
// Propagation.
// ===========================================================================
namespace {

struct Cand {
  uint64_t id, parent;
  double x[3], u[3];
  double E, s, s_max, h;
  int A, Z, q;
  double d_pion, d_pd, d_dec;
  bool states_drawn;
  uint32_t draws, events, generation, n_pion, n_pd, n_dropped;
  uint64_t n_acc, n_rej;
  int status;
  double x0[3], u0[3], E0;
  int A0, Z0;
};

struct Ctx {
  const orc_params* P;
  const double* grid;        // [nz][ny][nx][3]
  const double* t_beta;
  const double* t_pion;
  const double* t_gdr;
  double inv_spacing;
};

int64_t wrap_index(double fl, int64_t n) {
  int64_t i = (int64_t)fl % n;
  if (i < 0) i += n;
  return i;
}

double lerp(double a, double b, double t) { return a + t * (b - a); }

// Trilinear interpolation on the periodic vertex-centred grid: cell from
// floor((x - origin)/spacing) modulo N, then nested linear interpolation
// along x, then y, then z (reading: the paper stores fields on grids but does
// not state the interpolation).
void grid_field(const Ctx& C, const double x[3], double B[3]) {
  const orc_params& P = *C.P;
  int64_t i0[3], i1[3];
  double t[3];
  for (int d = 0; d < 3; ++d) {
    double r = (x[d] - P.origin[d]) * C.inv_spacing;
    double fl = std::floor(r);
    t[d] = r - fl;
    i0[d] = wrap_index(fl, P.n[d]);
    i1[d] = i0[d] + 1 == P.n[d] ? 0 : i0[d] + 1;
  }
  const int64_t nx = P.n[0], ny = P.n[1];
  auto at = [&](int64_t ix, int64_t iy, int64_t iz, int c) {
    return C.grid[((iz * ny + iy) * nx + ix) * 3 + c];
  };
  for (int c = 0; c < 3; ++c) {
    double c00 = lerp(at(i0[0], i0[1], i0[2], c), at(i1[0], i0[1], i0[2], c), t[0]);
    double c10 = lerp(at(i0[0], i1[1], i0[2], c), at(i1[0], i1[1], i0[2], c), t[0]);
    double c01 = lerp(at(i0[0], i0[1], i1[2], c), at(i1[0], i0[1], i1[2], c), t[0]);
    double c11 = lerp(at(i0[0], i1[1], i1[2], c), at(i1[0], i1[1], i1[2], c), t[0]);
    double c0 = lerp(c00, c10, t[1]);
    double c1_ = lerp(c01, c11, t[1]);
    B[c] = lerp(c0, c1_, t[2]);
  }
}

// Analytic regular galactic field (reading of the synthetic model "logarithmic
// spiral disk, pitch p, scale height h; toroidal halo"): galactocentric
// cylindrical coordinates (r, phi, z) about gal_center.
//   disk:  B = b_d exp(-|z|/h) (sin p r_hat + cos p phi_hat),  r_min <= r <= r_max
//   halo:  B_phi = b_h sign(z) exp(-(|z| - z0)^2 / (2 sigma^2))
void galactic_field(const orc_params& P, const double x[3], double B[3]) {
  double rx = x[0] - P.gal_center[0], ry = x[1] - P.gal_center[1], z = x[2] - P.gal_center[2];
  double r = std::sqrt(rx * rx + ry * ry);
  B[0] = 0.0; B[1] = 0.0; B[2] = 0.0;
  if (r == 0.0) return;
  double cr = rx / r, sr = ry / r;          // r_hat = (cr, sr), phi_hat = (-sr, cr)
  double az = std::fabs(z);
  double b_r = 0.0, b_phi = 0.0;
  if (r >= P.gal_disk_rmin && r <= P.gal_disk_rmax) {
    double bd = P.gal_disk_b * series_exp(-az / P.gal_disk_hz);
    b_r += bd * std::sin(P.gal_disk_pitch_rad);
    b_phi += bd * std::cos(P.gal_disk_pitch_rad);
  }
  if (z != 0.0) {
    double dz = az - P.gal_halo_z0;
    double bh = P.gal_halo_b * series_exp(-dz * dz / (2.0 * P.gal_halo_sigma * P.gal_halo_sigma));
    b_phi += z > 0.0 ? bh : -bh;
  }
  B[0] = b_r * cr - b_phi * sr;
  B[1] = b_r * sr + b_phi * cr;
}

// Analytic multi-arm galactic field of the Jansson-Farrar class (Sect. 4
// names analytic galactic models, JF12 among them; the structure follows
// R. Jansson and G. R. Farrar, ApJ 757:14, 2012, with the parameter values
// left to the caller).  Galactocentric cylindrical (r, phi, z) about
// gal_center, phi = atan2(y, x).  L(t, h, w) = 1 / (1 + exp(-2 (|t| - h) / w)).
//  * disk, times (1 - L(z, h_disk, w_disk)):
//      r_ring <= r < r_in:   B = ring_b phi_hat (molecular ring);
//      r_in <= r <= r_out:   B = arm_b[j] (r_in / r) (sin p r_hat + cos p phi_hat)
//    where j is the arm holding the logarithmic spiral through (r, phi): the
//    spiral's field lines obey d ln r / d phi = tan p, so it crosses phi = pi
//    at ln r_x = ln r + (pi - phi) tan p, and again at every multiple of
//    2 pi tan p; brought into [ln arm_rx[0], ln arm_rx[0] + 2 pi tan p), r_x
//    lies in [arm_rx[j], arm_rx[j+1]) (arm_rx[8] = arm_rx[0] e^{2 pi tan p}).
//  * toroidal halo: B_phi = e^{-|z|/halo_z0} L(z, h_disk, w_disk) times
//      halo_bn (1 - L(r, halo_rn, halo_wh)) for z >= 0,
//      halo_bs (1 - L(r, halo_rs, halo_wh)) for z < 0.
//  * X field: straight field lines in the (r, z) plane crossing the midplane
//    at r_p, of strength B_X(r_p) = x_b e^{-r_p / x_r} there, flux conserved
//    along each line.  Outside (r_p = r - |z| / tan x_theta >= x_rc) the lines
//    have elevation x_theta and |B| = B_X(r_p) r_p / r; inside, the line
//    through r_p has elevation atan(x_rc tan x_theta / r_p), so r_p = r f with
//    f = x_rc / (x_rc + |z| / tan x_theta), and |B| = B_X(r_p) f^2.
//    B_z = |B| sin(elevation), B_r = sign(z) |B| cos(elevation).
//  * zero where x^2 + y^2 + z^2 < r_cut_in^2 or > r_cut_out^2 (a cut of 0 is off);
//    on the axis r = 0 only B_z remains (reading).
double logistic(double t, double h, double w) {
  const double e = -2.0 * (std::fabs(t) - h) / w;
  if (e > 700.0) return 0.0;
  return 1.0 / (1.0 + series_exp(e));
}

int gmf_arm(const orc_gmf& G, double r, double phi) {
  const double tan_p = std::tan(G.pitch_rad);
  const double period = 2.0 * kPi * tan_p;
  const double ln_r0 = std::log(G.arm_rx[0]);
  double t = series_log(r) + (kPi - phi) * tan_p - ln_r0;
  t = t - std::floor(t / period) * period;
  if (t < 0.0) t = t + period;
  if (t >= period) t = t - period;
  int j = 7;
  while (j > 0 && t < std::log(G.arm_rx[j]) - ln_r0) --j;
  return j;
}

void gmf_field(const orc_params& P, const double x[3], double B[3]) {
  const orc_gmf& G = P.gmf;
  const double rx = x[0] - P.gal_center[0], ry = x[1] - P.gal_center[1];
  const double z = x[2] - P.gal_center[2];
  B[0] = 0.0; B[1] = 0.0; B[2] = 0.0;
  const double R2 = rx * rx + ry * ry + z * z;
  if (G.r_cut_in > 0.0 && R2 < G.r_cut_in * G.r_cut_in) return;
  if (G.r_cut_out > 0.0 && R2 > G.r_cut_out * G.r_cut_out) return;
  const double r = std::sqrt(rx * rx + ry * ry);
  const double az = std::fabs(z);
  const double l_disk = logistic(z, G.h_disk, G.w_disk);
  double b_r = 0.0, b_phi = 0.0, b_z = 0.0;
  if (r >= G.r_ring && r <= G.r_out && r > 0.0) {
    if (r < G.r_in) {
      b_phi += G.ring_b * (1.0 - l_disk);
    } else {
      const int j = gmf_arm(G, r, series_atan2(ry, rx));
      const double bd = G.arm_b[j] * (G.r_in / r) * (1.0 - l_disk);
      b_r += bd * std::sin(G.pitch_rad);
      b_phi += bd * std::cos(G.pitch_rad);
    }
  }
  const double bh = z >= 0.0 ? G.halo_bn * (1.0 - logistic(r, G.halo_rn, G.halo_wh))
                             : G.halo_bs * (1.0 - logistic(r, G.halo_rs, G.halo_wh));
  b_phi += series_exp(-az / G.halo_z0) * l_disk * bh;
  if (G.x_b != 0.0) {
    const double tan_t = std::tan(G.x_theta_rad);
    const double rp_out = r - az / tan_t;
    double bx, sin_e, cos_e;
    if (rp_out >= G.x_rc) {
      bx = G.x_b * series_exp(-rp_out / G.x_r) * (rp_out / r);
      sin_e = std::sin(G.x_theta_rad);
      cos_e = std::cos(G.x_theta_rad);
    } else {
      const double f = G.x_rc / (G.x_rc + az / tan_t);
      const double rp = r * f;
      bx = G.x_b * series_exp(-rp / G.x_r) * (f * f);
      const double q = G.x_rc * tan_t;  // tan(elevation) = q / r_p
      const double nrm = std::sqrt(rp * rp + q * q);
      sin_e = q / nrm;
      cos_e = rp / nrm;
    }
    b_z += bx * sin_e;
    if (z > 0.0) b_r += bx * cos_e;
    if (z < 0.0) b_r -= bx * cos_e;
  }
  if (r > 0.0) {
    const double cr = rx / r, sr = ry / r;  // r_hat = (cr, sr), phi_hat = (-sr, cr)
    B[0] = b_r * cr - b_phi * sr;
    B[1] = b_r * sr + b_phi * cr;
  }
  B[2] = b_z;
}

void field_at(const Ctx& C, const double x[3], double B[3]) {
  grid_field(C, x, B);
  if (C.P->flags & ORC_GALACTIC) {
    double G[3];
    galactic_field(*C.P, x, G);
    B[0] = B[0] + G[0];
    B[1] = B[1] + G[1];
    B[2] = B[2] + G[2];
  }
  if (C.P->flags & ORC_GMF) {
    double G[3];
    gmf_field(*C.P, x, G);
    B[0] = B[0] + G[0];
    B[1] = B[1] + G[1];
    B[2] = B[2] + G[2];
  }
}

// Equation of motion (reading: ultrarelativistic, s = c t, energy frozen
// during the step): dx/ds = u, du/ds = kappa (u x B), kappa = q Z c / E.
void rhs(const Ctx& C, const double y[6], double kappa, double k[6]) {
  double B[3];
  field_at(C, y, B);
  k[0] = y[3];
  k[1] = y[4];
  k[2] = y[5];
  double cx = y[4] * B[2] - y[5] * B[1];
  double cy = y[5] * B[0] - y[3] * B[2];
  double cz = y[3] * B[1] - y[4] * B[0];
  k[3] = kappa * cx;
  k[4] = kappa * cy;
  k[5] = kappa * cz;
}

double table_lookup(const Ctx& C, const double* tab, double lng) {
  const orc_params& P = *C.P;
  double t = (lng - P.tab_lg0) * P.tab_inv_dlg;
  double tmax = (double)(P.tab_n - 1);
  if (t < 0.0) t = 0.0;
  if (t > tmax) t = tmax;
  int64_t i = (int64_t)std::floor(t);
  if (i > P.tab_n - 2) i = P.tab_n - 2;
  double f = t - (double)i;
  return tab[i] + f * (tab[i + 1] - tab[i]);
}

double gamma_of(const Cand& c) { return c.E / ((double)c.A * kMpC2); }

double draw_uniform(const Ctx& C, Cand& c) {
  Words4 w = draw_words(C.P->seed, kTagInteraction, c.id, c.draws);
  c.draws += 1;
  return uniform_open(w.w[0], w.w[1]);
}

// Neutron decay length per eV of energy: c tau_n / (m_n c^2), in length units.
double decay_k(const orc_params& P) { return kC * kTauN / kMnC2 / P.length_unit_m; }

// Table entry of nuclide (A, Z) with A >= 2 ([tau, b_beta-, b_beta+, b_n, b_p]),
// or NULL when the table has none (stable).
const double* nuclide(const orc_params& P, int A, int Z) {
  if (!P.nuc_tab || A < 2 || A > P.nuc_amax || Z < 0 || Z > A) return nullptr;
  return P.nuc_tab + 5 * ((int64_t)A * (A + 1) / 2 + Z);
}

// Decay length per eV of energy of a nucleus of mass A m_p and lifetime tau:
// c tau / (A m_p c^2), in length units.
double nuc_decay_k(const orc_params& P, int A, double tau) {
  return kC * tau / ((double)A * kMpC2) / P.length_unit_m;
}

// Reset of all stochastic interaction states (Sect. 3: after an interaction
// the states of all interactions are reset).  Each state is the remaining
// free path d = -ln(u) / R(E), drawn at the candidate's current energy, in
// module-list order [pion production, photodisintegration].
void reset_states(const Ctx& C, Cand& c) {
  const orc_params& P = *C.P;
  double lng = series_log(gamma_of(c));
  if (P.flags & ORC_PION) {
    double u = draw_uniform(C, c);
    double R = (double)c.A * table_lookup(C, C.t_pion, lng);
    c.d_pion = R > 0.0 ? -series_log(u) / R : INFINITY;
  }
  if (P.flags & ORC_PHOTODIS) {
    double u = draw_uniform(C, c);
    double R = c.A >= 2 ? (double)c.A * table_lookup(C, C.t_gdr, lng) : 0.0;
    c.d_pd = R > 0.0 ? -series_log(u) / R : INFINITY;
  }
  if (P.flags & ORC_DECAY) {
    // free neutrons: decay length gamma c tau = (E / m_n c^2) c tau (reading:
    // the uniform is drawn for every species, so draw counts depend on the
    // module list only); an unstable nucleus of the table: gamma c tau with
    // gamma = E / (A m_p c^2)
    double u = draw_uniform(C, c);
    if (c.A == 1 && c.Z == 0) {
      c.d_dec = -series_log(u) * (c.E * decay_k(P));
    } else {
      const double* e = nuclide(P, c.A, c.Z);
      c.d_dec = (e && std::isfinite(e[0])) ? -series_log(u) * (c.E * nuc_decay_k(P, c.A, e[0]))
                                           : INFINITY;
    }
  }
  c.states_drawn = true;
}

// Does the segment a -> b enter the sphere (centre cen, radius R) from outside?
bool segment_enters(const double a[3], const double b[3], const double cen[3], double R) {
  double f[3], d[3], g[3];
  for (int i = 0; i < 3; ++i) {
    f[i] = a[i] - cen[i];
    d[i] = b[i] - a[i];
    g[i] = b[i] - cen[i];
  }
  double R2 = R * R;
  double fa = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
  if (fa <= R2) return false;                       // started inside
  double gb = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  if (gb <= R2) return true;                        // ends inside
  double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (dd == 0.0) return false;
  double fd = f[0] * d[0] + f[1] * d[1] + f[2] * d[2];
  double tstar = -fd / dd;                          // closest approach on the line
  if (!(tstar > 0.0 && tstar < 1.0)) return false;
  double m2 = fa - fd * fd / dd;                    // squared closest distance
  return m2 <= R2;
}

Cand make_secondary(const Cand& p, int A, int Z, double E, double h_max) {
  Cand s;
  std::memset(&s, 0, sizeof(s));
  s.id = child_id(p.id, p.events);
  s.parent = p.id;
  for (int i = 0; i < 3; ++i) {
    s.x[i] = p.x[i];
    s.u[i] = p.u[i];
    s.x0[i] = p.x[i];
    s.u0[i] = p.u[i];
  }
  s.E = E;
  s.E0 = E;
  s.s = p.s;
  s.s_max = p.s_max;
  s.h = h_max;
  s.A = A; s.Z = Z; s.q = p.q;
  s.A0 = A; s.Z0 = Z;
  s.states_drawn = false;
  s.generation = p.generation + 1;
  s.status = ORC_ACTIVE;
  return s;
}

// One candidate, all module cycles until IsActive is false.  Secondaries are
// appended to `out_secondaries`.
void propagate_one(const Ctx& C, Cand& c, std::vector<Cand>& out_secondaries) {
  const orc_params& P = *C.P;
  const bool pion_on = (P.flags & ORC_PION) != 0;
  const bool pd_on = (P.flags & ORC_PHOTODIS) != 0;
  const bool dec_on = (P.flags & ORC_DECAY) != 0;
  while (c.status == ORC_ACTIVE) {
    if ((pion_on || pd_on || dec_on) && !c.states_drawn) reset_states(C, c);
    // ---- integration module: Cash-Karp trial steps until accepted ----
    double h = c.h;
    if (h > P.h_max) h = P.h_max;
    const double cap_s = c.s_max - c.s;
    if (cap_s < h) h = cap_s;
    if (pion_on && c.d_pion < h) h = c.d_pion;
    if (pd_on && c.d_pd < h) h = c.d_pd;
    if (dec_on && c.d_dec < h) h = c.d_dec;
    const double kappa = (double)(c.q * c.Z) * P.curv_k / c.E;
    double y[6] = {c.x[0], c.x[1], c.x[2], c.u[0], c.u[1], c.u[2]};
    double k1[6], k2[6], k3[6], k4[6], k5[6], k6[6], yt[6], y5[6];
    rhs(C, y, kappa, k1);
    double eps;
    int rejections = 0;
    for (;;) {
      for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (b21 * k1[i]);
      rhs(C, yt, kappa, k2);
      for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (b31 * k1[i] + b32 * k2[i]);
      rhs(C, yt, kappa, k3);
      for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (b41 * k1[i] + b42 * k2[i] + b43 * k3[i]);
      rhs(C, yt, kappa, k4);
      for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (b51 * k1[i] + b52 * k2[i] + b53 * k3[i] + b54 * k4[i]);
      rhs(C, yt, kappa, k5);
      for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (b61 * k1[i] + b62 * k2[i] + b63 * k3[i] + b64 * k4[i] + b65 * k5[i]);
      rhs(C, yt, kappa, k6);
      for (int i = 0; i < 6; ++i)
        y5[i] = y[i] + h * (c1 * k1[i] + c3 * k3[i] + c4 * k4[i] + c6 * k6[i]);
      double err[3];
      for (int i = 0; i < 3; ++i)
        err[i] = h * (e1 * k1[3 + i] + e3 * k3[3 + i] + e4 * k4[3 + i] + e5 * k5[3 + i] +
                      e6 * k6[3 + i]);
      // error norm on the direction (dimensionless, |u| = 1): relative error
      eps = std::sqrt(err[0] * err[0] + err[1] * err[1] + err[2] * err[2]) / P.tol;
      if (eps <= 1.0 || h <= P.h_min || rejections >= 64) break;
      // reject: shrink by 0.95 eps^(-1/4), at most tenfold, not below h_min
      double fac = 0.95 / std::sqrt(std::sqrt(eps));
      if (fac < 0.1) fac = 0.1;
      double hn = h * fac;
      if (hn < P.h_min) hn = P.h_min;
      h = hn;
      rejections += 1;
      c.n_rej += 1;
    }
    // accept
    double x_old[3] = {c.x[0], c.x[1], c.x[2]};
    c.x[0] = y5[0]; c.x[1] = y5[1]; c.x[2] = y5[2];
    double un = std::sqrt(y5[3] * y5[3] + y5[4] * y5[4] + y5[5] * y5[5]);
    double inv = 1.0 / un;
    c.u[0] = y5[3] * inv; c.u[1] = y5[4] * inv; c.u[2] = y5[5] * inv;
    c.s = (h == cap_s) ? c.s_max : c.s + h;
    double grow = eps == 0.0 ? 5.0 : 0.95 / std::sqrt(std::sqrt(eps));
    if (grow > 5.0) grow = 5.0;
    double h_next = h * grow;
    if (h_next < P.h_min) h_next = P.h_min;
    if (h_next > P.h_max) h_next = P.h_max;
    c.h = h_next;
    c.n_acc += 1;
    // ---- continuous losses: pair production (CMB) and adiabatic ----
    if (P.flags & (ORC_PAIR | ORC_ADIABATIC)) {
      double beta = 0.0;
      if (P.flags & ORC_PAIR) {
        double bp = table_lookup(C, C.t_beta, series_log(gamma_of(c)));
        beta = bp * (double)(c.Z * c.Z) / (double)c.A;
      }
      if (P.flags & ORC_ADIABATIC) beta = beta + P.beta_ad;
      c.E = c.E * (1.0 - beta * h);
    }
    // ---- stochastic interactions: decrement, first in list fires ----
    if (pion_on || pd_on || dec_on) {
      if (pion_on) c.d_pion = c.d_pion - h;
      if (pd_on) c.d_pd = c.d_pd - h;
      if (dec_on) c.d_dec = c.d_dec - h;
      if (pion_on && c.d_pion <= 0.0) {
        // photo-pion event (reading): one nucleon loses inelasticity 0.2
        c.E = c.E - 0.2 * c.E / (double)c.A;
        c.n_pion += 1;
        c.events += 1;
        reset_states(C, c);
      } else if (pd_on && c.d_pd <= 0.0) {
        // single-nucleon emission (reading): proton with probability Z/A,
        // kept away from Z' = 0 or N' = 0 daughters with A' >= 2
        double u = draw_uniform(C, c);
        bool proton = u < (double)c.Z / (double)c.A;
        int Ad = c.A - 1;
        if (proton && Ad >= 2 && c.Z - 1 == 0) proton = false;
        if (!proton && Ad >= 2 && Ad - c.Z == 0) proton = true;
        double En = c.E / (double)c.A;
        double Ed = c.E * (double)Ad / (double)c.A;
        Cand sec = make_secondary(c, 1, proton ? 1 : 0, En, P.h_max);
        if (!(P.flags & ORC_EMIN) || En >= P.e_min)
          out_secondaries.push_back(sec);
        else
          c.n_dropped += 1;
        c.A = Ad;
        c.Z = c.Z - (proton ? 1 : 0);
        c.E = Ed;
        c.n_pd += 1;
        c.events += 1;
        reset_states(C, c);
      } else if (dec_on && c.d_dec <= 0.0) {
        if (c.A == 1 && c.Z == 0) {
          // beta decay n -> p e nu (reading): the proton keeps the Lorentz
          // factor; electron and antineutrino are not followed
          c.Z = 1;
          c.E = c.E * (kMpC2 / kMnC2);
        } else {
          // unstable nucleus (reading): the channel is the first whose
          // cumulative branching fraction exceeds a uniform draw (order
          // beta-, beta+, n, p; past the last sum, the last channel with a
          // non-zero fraction).  beta-+: Z +- 1, the nucleus (mass A m_p)
          // keeps its energy, the leptons are not followed.  Nucleon
          // emission: as in photodisintegration, the nucleon carries E / A
          // and the daughter E (A - 1) / A.
          const double* e = nuclide(P, c.A, c.Z);
          double u = draw_uniform(C, c);
          int ch = -1, last = 0;
          double acc = 0.0;
          for (int k = 0; k < 4; ++k) {
            acc = acc + e[1 + k];
            if (e[1 + k] > 0.0) last = k;
            if (ch < 0 && u < acc) ch = k;
          }
          if (ch < 0) ch = last;
          if (ch == 0) {
            c.Z = c.Z + 1;
          } else if (ch == 1) {
            c.Z = c.Z - 1;
          } else {
            const bool proton = ch == 3;
            const int Ad = c.A - 1;
            double En = c.E / (double)c.A;
            double Ed = c.E * (double)Ad / (double)c.A;
            Cand sec = make_secondary(c, 1, proton ? 1 : 0, En, P.h_max);
            if (!(P.flags & ORC_EMIN) || En >= P.e_min)
              out_secondaries.push_back(sec);
            else
              c.n_dropped += 1;
            c.A = Ad;
            c.Z = c.Z - (proton ? 1 : 0);
            c.E = Ed;
          }
        }
        c.events += 1;
        reset_states(C, c);
      }
    }
    // ---- break conditions: minimum energy, trajectory length, observer, border ----
    if ((P.flags & ORC_EMIN) && c.E < P.e_min) {
      c.status = ORC_BELOW_EMIN;
    } else if (c.s >= c.s_max) {
      c.status = ORC_MAX_LENGTH;
    } else if ((P.flags & ORC_OBSERVER) && segment_enters(x_old, c.x, P.obs_c, P.obs_r)) {
      c.status = ORC_DETECTED;
    } else if (P.flags & ORC_BORDER) {
      double dx = c.x[0] - P.border_c[0], dy = c.x[1] - P.border_c[1], dz = c.x[2] - P.border_c[2];
      if (dx * dx + dy * dy + dz * dz >= P.border_r * P.border_r) c.status = ORC_AT_BORDER;
    }
    if (c.status == ORC_ACTIVE && (int64_t)c.n_acc >= P.max_steps) c.status = ORC_BUDGET;
  }
}

void to_record(const Cand& c, orc_record& r) {
  std::memset(&r, 0, sizeof(r));
  r.id = c.id; r.parent_id = c.parent;
  for (int i = 0; i < 3; ++i) {
    r.x[i] = c.x[i]; r.u[i] = c.u[i]; r.x0[i] = c.x0[i]; r.u0[i] = c.u0[i];
  }
  r.E = c.E; r.s = c.s; r.E0 = c.E0; r.s_max = c.s_max;
  r.n_acc = c.n_acc; r.n_rej = c.n_rej;
  r.A = c.A; r.Z = c.Z; r.A0 = c.A0; r.Z0 = c.Z0; r.q = c.q;
  r.status = c.status;
  r.n_pion = c.n_pion; r.n_pd = c.n_pd; r.draws = c.draws; r.generation = c.generation;
  r.n_dropped = c.n_dropped;
}

}  // namespace

extern "C" {

// Propagate n primaries and, depth first, every secondary they spawn.
// Records are written in primary order, each primary followed by its
// descendants.  Returns 0 on success, -1 if out_cap was too small (n_out then
// holds the count needed), -2 on invalid arguments.
int orc_propagate(const orc_params* P, const double* grid, const double* t_beta,
                  const double* t_pion, const double* t_gdr, int64_t n, const uint64_t* id,
                  const double* x, const double* y, const double* z, const double* ux,
                  const double* uy, const double* uz, const double* E, const double* s_max,
                  const int32_t* A, const int32_t* Z, const int32_t* q, orc_record* out,
                  int64_t out_cap, int64_t* n_out, int nthreads) {
  if (!P || !grid || n < 0 || !n_out) return -2;
  Ctx C;
  C.P = P; C.grid = grid; C.t_beta = t_beta; C.t_pion = t_pion; C.t_gdr = t_gdr;
  C.inv_spacing = 1.0 / P->spacing;
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<orc_record>> per(n);
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    std::vector<Cand> stack;
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= n) break;
      Cand c;
      std::memset(&c, 0, sizeof(c));
      c.id = id[i];
      c.parent = 0;
      c.x[0] = x[i]; c.x[1] = y[i]; c.x[2] = z[i];
      c.u[0] = ux[i]; c.u[1] = uy[i]; c.u[2] = uz[i];
      for (int d = 0; d < 3; ++d) { c.x0[d] = c.x[d]; c.u0[d] = c.u[d]; }
      c.E = E[i]; c.E0 = E[i];
      c.s = 0.0;
      c.s_max = s_max ? s_max[i] : INFINITY;
      c.h = P->h_max;
      c.A = A[i]; c.Z = Z[i]; c.q = q ? q[i] : 1;
      c.A0 = c.A; c.Z0 = c.Z;
      c.status = ORC_ACTIVE;
      stack.clear();
      stack.push_back(c);
      std::vector<orc_record>& dst = per[i];
      while (!stack.empty()) {
        Cand cur = stack.front();
        stack.erase(stack.begin());
        std::vector<Cand> secs;
        propagate_one(C, cur, secs);
        orc_record r;
        to_record(cur, r);
        dst.push_back(r);
        for (auto& s : secs) stack.push_back(s);
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  int64_t total = 0;
  for (auto& v : per) total += (int64_t)v.size();
  *n_out = total;
  if (total > out_cap) return -1;
  int64_t k = 0;
  for (auto& v : per)
    for (auto& r : v) out[k++] = r;
  return 0;
}

}  // extern "C"

extern "C" {

// Table axis: ln(Gamma) of node 0 and nodes per unit ln(Gamma).
void orc_table_axis(int64_t n, double g_lo, double g_hi, double* lg0, double* inv_dlg) {
  *lg0 = std::log(g_lo);
  *inv_dlg = (double)(n - 1) / (std::log(g_hi) - std::log(g_lo));
}

// Field at a list of points (grid interpolation, plus the analytic galactic
// field when its flag is set); used by the interpolation pins.
void orc_field_at(const orc_params* P, const double* grid, int64_t n, const double* pts,
                  double* out) {
  Ctx C;
  std::memset(&C, 0, sizeof(C));
  C.P = P;
  C.grid = grid;
  C.inv_spacing = 1.0 / P->spacing;
  for (int64_t i = 0; i < n; ++i) field_at(C, pts + 3 * i, out + 3 * i);
}

}  // extern "C"

// ===========================================================================
// 1D mode with cosmology and the a-posteriori 3D cosmology correction
// (Sect. 2 lists the 1D mode with cosmological effects; Sect. 4 "Cosmology in
// 3D" gives the correction).  Readings, each stated once here:
//  * flat Lambda-CDM: H(z) = H0 sqrt(Om (1+z)^3 + OL); lengths comoving;
//  * the candidate moves toward the observer, its redshift falling to 0; a
//    step is a redshift decrement dz, its comoving length dz / H(z - dz/2)
//    (midpoint rule; H per length unit, i.e. H/c);
//  * adiabatic loss: the exact redshift factor E <- E (1+z') / (1+z);
//  * pair loss and interaction rates from the z = 0 tables: per comoving
//    length (1+z)^2 rate((1+z) Gamma) (photon density (1+z)^3, energies
//    (1+z), proper length = comoving / (1+z)); neutron decay 1 / ((1+z)
//    gamma c tau);
//  * stochastic states are remaining optical depths tau = -ln(u), reduced by
//    rate * length; a step is capped where a depth would run out (the event
//    then happens at its end), by dz_max, by a relative pair loss loss_max,
//    and by z itself;
//  * events, secondaries and lineage ids as in 3D; arrival at z = 0 is
//    status "detected";
//  * the correction places the 1D source at the redshift whose comoving
//    distance is the 3D trajectory length (3D coordinates are comoving).
// ===========================================================================
struct orc_params1d {
  uint32_t flags;     // ORC_PAIR | ORC_ADIABATIC | ORC_PION | ORC_PHOTODIS | ORC_EMIN | ORC_DECAY
  uint32_t pad0;
  uint64_t seed;
  double e_min;       // [eV]
  double H0;          // Hubble constant / c [1 / length unit]
  double omega_m, omega_l;
  double dz_max;      // largest redshift step
  double loss_max;    // largest relative pair loss per step
  double tab_lg0, tab_inv_dlg;
  int64_t tab_n;
  double length_unit_m;
  int64_t max_steps;
};

namespace {

const uint32_t kTagCosmology = 5;

struct Ctx1d {
  const orc_params1d* P;
  const double* t_beta;
  const double* t_pion;
  const double* t_gdr;
};

double hubble(const orc_params1d& P, double z) {
  const double a = 1.0 + z;
  return P.H0 * std::sqrt(P.omega_m * a * a * a + P.omega_l);
}

double lookup1d(const orc_params1d& P, const double* tab, double lng) {
  double t = (lng - P.tab_lg0) * P.tab_inv_dlg;
  double tmax = (double)(P.tab_n - 1);
  if (t < 0.0) t = 0.0;
  if (t > tmax) t = tmax;
  int64_t i = (int64_t)std::floor(t);
  if (i > P.tab_n - 2) i = P.tab_n - 2;
  double f = t - (double)i;
  return tab[i] + f * (tab[i + 1] - tab[i]);
}

double draw1d(const Ctx1d& C, Cand& c) {
  Words4 w = draw_words(C.P->seed, kTagInteraction, c.id, c.draws);
  c.draws += 1;
  return uniform_open(w.w[0], w.w[1]);
}

// optical depths in module order [pion, photodisintegration, decay]
void reset1d(const Ctx1d& C, Cand& c) {
  const uint32_t f = C.P->flags;
  if (f & ORC_PION) c.d_pion = -series_log(draw1d(C, c));
  if (f & ORC_PHOTODIS) c.d_pd = -series_log(draw1d(C, c));
  if (f & ORC_DECAY) c.d_dec = -series_log(draw1d(C, c));
  c.states_drawn = true;
}

struct Rates1d {
  double beta, pion, pd, dec;  // per comoving length
};

Rates1d rates1d(const Ctx1d& C, const Cand& c, double z) {
  const orc_params1d& P = *C.P;
  Rates1d r = {0.0, 0.0, 0.0, 0.0};
  const double a = 1.0 + z;
  const double lng = series_log(a * gamma_of(c));
  if (P.flags & ORC_PAIR)
    r.beta = a * a * lookup1d(P, C.t_beta, lng) * (double)(c.Z * c.Z) / (double)c.A;
  if (P.flags & ORC_PION) r.pion = a * a * (double)c.A * lookup1d(P, C.t_pion, lng);
  if ((P.flags & ORC_PHOTODIS) && c.A >= 2)
    r.pd = a * a * (double)c.A * lookup1d(P, C.t_gdr, lng);
  if ((P.flags & ORC_DECAY) && c.A == 1 && c.Z == 0) {
    const double k = kC * kTauN / kMnC2 / P.length_unit_m;
    r.dec = 1.0 / (a * c.E * k);
  }
  return r;
}

void propagate_one_1d(const Ctx1d& C, Cand& c, std::vector<Cand>& out_secondaries) {
  const orc_params1d& P = *C.P;
  const bool pion_on = (P.flags & ORC_PION) != 0;
  const bool pd_on = (P.flags & ORC_PHOTODIS) != 0;
  const bool dec_on = (P.flags & ORC_DECAY) != 0;
  while (c.status == ORC_ACTIVE) {
    if ((pion_on || pd_on || dec_on) && !c.states_drawn) reset1d(C, c);
    const double z = c.x[0];
    const Rates1d r = rates1d(C, c, z);
    const double H = hubble(P, z);
    // redshift step: the smallest cap (0: none, 1: z, 2: pion, 3: pd, 4: decay)
    double dz = P.dz_max;
    int cap = 0;
    if (r.beta > 0.0 && P.loss_max * H / r.beta < dz) dz = P.loss_max * H / r.beta;
    if (z <= dz) {
      dz = z;
      cap = 1;
    }
    if (pion_on && r.pion > 0.0 && c.d_pion * H / r.pion < dz) {
      dz = c.d_pion * H / r.pion;
      cap = 2;
    }
    if (pd_on && r.pd > 0.0 && c.d_pd * H / r.pd < dz) {
      dz = c.d_pd * H / r.pd;
      cap = 3;
    }
    if (dec_on && r.dec > 0.0 && c.d_dec * H / r.dec < dz) {
      dz = c.d_dec * H / r.dec;
      cap = 4;
    }
    const double z1 = cap == 1 ? 0.0 : z - dz;
    const double h = dz / hubble(P, z - 0.5 * dz);  // comoving length of the step
    // continuous losses: pair (explicit, start-of-step rate), then the exact
    // adiabatic redshift factor
    if (P.flags & ORC_PAIR) c.E = c.E * (1.0 - r.beta * h);
    if (P.flags & ORC_ADIABATIC) c.E = c.E * ((1.0 + z1) / (1.0 + z));
    c.x[0] = z1;
    c.s = c.s + h;
    c.n_acc += 1;
    // optical depths
    if (pion_on) c.d_pion = cap == 2 ? 0.0 : c.d_pion - r.pion * h;
    if (pd_on) c.d_pd = cap == 3 ? 0.0 : c.d_pd - r.pd * h;
    if (dec_on) c.d_dec = cap == 4 ? 0.0 : c.d_dec - r.dec * h;
    if (pion_on && c.d_pion <= 0.0) {
      c.E = c.E - 0.2 * c.E / (double)c.A;
      c.n_pion += 1;
      c.events += 1;
      reset1d(C, c);
    } else if (pd_on && c.A >= 2 && c.d_pd <= 0.0) {
      double u = draw1d(C, c);
      bool proton = u < (double)c.Z / (double)c.A;
      int Ad = c.A - 1;
      if (proton && Ad >= 2 && c.Z - 1 == 0) proton = false;
      if (!proton && Ad >= 2 && Ad - c.Z == 0) proton = true;
      double En = c.E / (double)c.A;
      double Ed = c.E * (double)Ad / (double)c.A;
      Cand sec = make_secondary(c, 1, proton ? 1 : 0, En, 0.0);
      sec.x[0] = c.x[0];
      sec.x0[0] = c.x[0];
      if (!(P.flags & ORC_EMIN) || En >= P.e_min)
        out_secondaries.push_back(sec);
      else
        c.n_dropped += 1;
      c.A = Ad;
      c.Z = c.Z - (proton ? 1 : 0);
      c.E = Ed;
      c.n_pd += 1;
      c.events += 1;
      reset1d(C, c);
    } else if (dec_on && c.A == 1 && c.Z == 0 && c.d_dec <= 0.0) {
      c.Z = 1;
      c.E = c.E * (kMpC2 / kMnC2);
      c.events += 1;
      reset1d(C, c);
    }
    if ((P.flags & ORC_EMIN) && c.E < P.e_min)
      c.status = ORC_BELOW_EMIN;
    else if (c.x[0] <= 0.0)
      c.status = ORC_DETECTED;
    if (c.status == ORC_ACTIVE && (int64_t)c.n_acc >= P.max_steps) c.status = ORC_BUDGET;
  }
}

// Comoving distance (length units) to redshift z: integral of dz' / H(z')
// (H per length unit) by composite Simpson with 4096 panels.
double comoving_distance(const orc_params1d& P, double z) {
  const int n = 4096;
  const double w = z / n;
  auto f = [&](double x) { return 1.0 / hubble(P, x); };
  double sum = f(0.0) + f(z);
  for (int i = 1; i < n; ++i) sum += (i % 2 ? 4.0 : 2.0) * f(i * w);
  return sum * w / 3.0;
}

}  // namespace

extern "C" {

// 1D propagation of n primaries from redshifts z_src (and every secondary,
// depth first).  Records: x[0] = final redshift, x0[0] = starting redshift,
// s = comoving length travelled, u = 0.  Return codes as orc_propagate.
int orc_propagate_1d(const orc_params1d* P, const double* t_beta, const double* t_pion,
                     const double* t_gdr, int64_t n, const uint64_t* id, const double* z_src,
                     const double* E, const int32_t* A, const int32_t* Z, orc_record* out,
                     int64_t out_cap, int64_t* n_out, int nthreads) {
  if (!P || n < 0 || !n_out) return -2;
  Ctx1d C = {P, t_beta, t_pion, t_gdr};
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<orc_record>> per(n);
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    std::vector<Cand> stack;
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= n) break;
      Cand c;
      std::memset(&c, 0, sizeof(c));
      c.id = id[i];
      c.x[0] = z_src[i];
      c.x0[0] = z_src[i];
      c.E = E[i];
      c.E0 = E[i];
      c.A = A[i];
      c.Z = Z[i];
      c.A0 = A[i];
      c.Z0 = Z[i];
      c.q = 1;
      c.status = ORC_ACTIVE;
      stack.clear();
      stack.push_back(c);
      while (!stack.empty()) {
        Cand cur = stack.back();
        stack.pop_back();
        std::vector<Cand> secs;
        propagate_one_1d(C, cur, secs);
        orc_record r;
        to_record(cur, r);
        per[i].push_back(r);
        for (auto& s : secs) stack.push_back(s);
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  int64_t total = 0;
  for (auto& v : per) total += (int64_t)v.size();
  *n_out = total;
  if (total > out_cap) return -1;
  int64_t k = 0;
  for (auto& v : per)
    for (auto& r : v) out[k++] = r;
  return 0;
}

// Comoving distance (length units) to each redshift.
void orc_comoving_distance(const orc_params1d* P, int64_t n, const double* z, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = comoving_distance(*P, z[i]);
}

// Redshift at comoving distance D (bisection to 1e-15 relative).
void orc_redshift_of_distance(const orc_params1d* P, int64_t n, const double* D, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    double lo = 0.0, hi = 1.0;
    while (comoving_distance(*P, hi) < D[i] && hi < 1e6) hi *= 2.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
      double mid = 0.5 * (lo + hi);
      if (comoving_distance(*P, mid) < D[i])
        lo = mid;
      else
        hi = mid;
    }
    out[i] = 0.5 * (lo + hi);
  }
}

// The a-posteriori correction (Sect. 4): particle i (id, injected E, A, Z)
// is re-propagated in 1D from redshift z_src[i]; of its products that reach
// z = 0, ordered by id, product k = min(floor(u n_k), n_k - 1) is taken, u
// from Philox tag 5, counter (0, id).  Outputs its E, A, Z and n_k (0: no
// product reaches the observer; E, A, Z then 0).
int orc_cosmology_pick(const orc_params1d* P, const double* t_beta, const double* t_pion,
                       const double* t_gdr, int64_t n, const uint64_t* id, const double* z_src,
                       const double* E, const int32_t* A, const int32_t* Z, double* E_out,
                       int32_t* A_out, int32_t* Z_out, int32_t* n_products, int nthreads) {
  if (!P || n < 0) return -2;
  Ctx1d C = {P, t_beta, t_pion, t_gdr};
  if (nthreads < 1) nthreads = 1;
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    std::vector<Cand> stack;
    std::vector<Cand> arrived;
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= n) break;
      Cand c;
      std::memset(&c, 0, sizeof(c));
      c.id = id[i];
      c.x[0] = z_src[i];
      c.x0[0] = z_src[i];
      c.E = E[i];
      c.E0 = E[i];
      c.A = A[i];
      c.Z = Z[i];
      c.A0 = A[i];
      c.Z0 = Z[i];
      c.q = 1;
      c.status = ORC_ACTIVE;
      stack.clear();
      arrived.clear();
      stack.push_back(c);
      while (!stack.empty()) {
        Cand cur = stack.back();
        stack.pop_back();
        std::vector<Cand> secs;
        propagate_one_1d(C, cur, secs);
        if (cur.status == ORC_DETECTED) arrived.push_back(cur);
        for (auto& s : secs) stack.push_back(s);
      }
      std::sort(arrived.begin(), arrived.end(),
                [](const Cand& a, const Cand& b) { return a.id < b.id; });
      const int64_t nk = (int64_t)arrived.size();
      n_products[i] = (int32_t)nk;
      if (nk == 0) {
        E_out[i] = 0.0;
        A_out[i] = 0;
        Z_out[i] = 0;
        continue;
      }
      Words4 w = draw_words(P->seed, kTagCosmology, c.id, 0);
      const double u = uniform_open(w.w[0], w.w[1]);
      int64_t k = (int64_t)std::floor(u * (double)nk);
      if (k > nk - 1) k = nk - 1;
      E_out[i] = arrived[k].E;
      A_out[i] = arrived[k].A;
      Z_out[i] = arrived[k].Z;
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return 0;
}

}  // extern "C"
