// tables.cu -- interaction-rate tables computed on the device.
//
// Node i of n sits at ln(Gamma_i) = ln(gamma_lo) + i (ln gamma_hi - ln gamma_lo)/(n-1).
// One thread per node evaluates
//   beta_pair  Blumenthal (Phys. Rev. D 1, 1596, 1970) energy-loss rate of a
//              proton on a Planck photon gas,
//                (1/E) dE/dx = alpha r_e^2 (m_e c^2)^2 / (Gamma m_p c^2)
//                              * int_2^inf dk n(k m_e c^2 / 2 Gamma) phi(k) / k^2,
//              with phi(k) from the fit of Chodorowski, Zdziarski & Sikora
//              (ApJ 400, 181, 1992);
//   rate_pion  the photo-pion rate of a nucleon for a step cross section,
//              which for a Planck gas is the Bose-Einstein series
//                R = 2 sigma0 (kT/hbar c)^3 / pi^2 sum_n e^{-n x0} (x0/n^2 + 1/n^3),
//              x0 = eps_th / (2 Gamma kT);
//   rate_gdr   the photodisintegration rate per nucleon for a Lorentzian
//              giant dipole resonance cut to [lo, hi],
//                R = 1/(2 Gamma^2) int d eps n(eps)/eps^2 int_lo^{min(2 Gamma eps, hi)} e' sigma(e') de'
//              with the inner integral in closed form.
// Quadrature: composite 32-point Gauss-Legendre in the logarithm of the
// integration variable, with breakpoints where the integrand has a kink.
#include <math.h>

#include <vector>

#include "crp_internal.cuh"
#include "field_internal.h"

namespace crp {

namespace {

constexpr int kGL = 32;
constexpr int kPanels = 64;

// Gauss-Legendre rule on [-1, 1], computed on the host and passed to the
// kernel by value (no per-device state to initialise).
struct GLRule {
  double x[kGL], w[kGL];
};

// Physical constants (CODATA 2018).
constexpr double kMe = 0.51099895000e6;        // m_e c^2 [eV]
constexpr double kMp = 938.27208816e6;         // m_p c^2 [eV]
constexpr double kAlphaFS = 7.2973525693e-3;
constexpr double kRe = 2.8179403262e-15;       // [m]
constexpr double kBoltz = 8.617333262e-5;      // [eV/K]
constexpr double kHC = 1.973269804e-7;         // hbar c [eV m]

// Photon number density of a Planck spectrum per unit energy [1 / (m^3 eV)].
__device__ double planck(double eps, double kT) {
  const double x = eps / kT;
  if (x > 700.0) return 0.0;
  const double hc3 = kHC * kHC * kHC;
  return eps * eps / (M_PI * M_PI * hc3 * expm1(x));
}

// Chodorowski et al. (1992) approximation of Blumenthal's phi(kappa).
__device__ double phi_cz(double k) {
  if (k <= 2.0) return 0.0;
  if (k < 25.0) {
    const double t = k - 2.0;
    const double t2 = t * t;
    const double poly = 1.0 + t * (0.8048 + t * (0.1459 + t * (1.137e-3 - 3.879e-6 * t)));
    return (M_PI / 12.0) * t2 * t2 / poly;
  }
  const double L = log(k);
  const double cubic = -86.07 + L * (50.96 + L * (-14.45 + L * (8.0 / 3.0)));
  const double corr = 1.0 - (2.910 + (78.35 + 1837.0 / k) / k) / k;
  return k * cubic / corr;
}

// Composite Gauss-Legendre on [a, b] with kPanels equal panels.
template <class F>
__device__ double gl_composite(const GLRule& gl, const F& f, double a, double b) {
  if (!(b > a)) return 0.0;
  const double w = (b - a) / kPanels;
  double total = 0.0;
  for (int p = 0; p < kPanels; ++p) {
    const double mid = a + (p + 0.5) * w, half = 0.5 * w;
    double s = 0.0;
    for (int j = 0; j < kGL; ++j) s += gl.w[j] * f(mid + half * gl.x[j]);
    total += s * half;
  }
  return total;
}

__device__ double beta_pair_dev(const GLRule& gl, double gamma, double kT) {
  const double kmax = 1400.0 * gamma * kT / kMe;  // Planck factor below e^-700 beyond
  if (kmax <= 2.0) return 0.0;
  auto g = [&](double y) {
    const double k = exp(y);
    return planck(k * kMe / (2.0 * gamma), kT) * phi_cz(k) / k;  // k * n * phi / k^2
  };
  const double lo = log(2.0), mid = log(25.0), hi = log(kmax);
  const double I = hi <= mid ? gl_composite(gl, g, lo, hi)
                             : gl_composite(gl, g, lo, mid) + gl_composite(gl, g, mid, hi);
  return kAlphaFS * kRe * kRe * kMe * kMe * I / (gamma * kMp);
}

__device__ double rate_pion_dev(double gamma, double kT, double sigma0, double eth) {
  const double x0 = eth / (2.0 * gamma * kT);
  double sum = 0.0;
  for (int n = 1; n < 200000; ++n) {
    const double e = exp(-(double)n * x0);
    if (e == 0.0) break;
    const double dn = (double)n;
    const double term = e * (x0 / (dn * dn) + 1.0 / (dn * dn * dn));
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  const double t = kT / kHC;
  return 2.0 * sigma0 * t * t * t * sum / (M_PI * M_PI);
}

// int_lo^{min(e, hi)} e' sigma(e') de' for the Lorentzian, without
// cancellation near the lower limit.
__device__ double gdr_inner_dev(double e, double peak, double ec, double w, double lo, double hi) {
  if (e <= lo) return 0.0;
  const double top = e < hi ? e : hi;
  const double D = top - lo, a = lo - ec, b = top - ec;
  const double logs = 0.5 * log1p(D * (a + b) / (a * a + w * w));
  const double ang = (ec / w) * atan2(w * D, w * w + a * b);
  return peak * w * w * (logs + ang);
}

__device__ double rate_gdr_dev(const GLRule& gl, double gamma, double kT, double peak, double ec,
                               double w, double lo, double hi) {
  const double e_lo = lo / (2.0 * gamma), e_hi = 700.0 * kT;
  if (e_hi <= e_lo) return 0.0;
  auto g = [&](double y) {
    const double eps = exp(y);
    return planck(eps, kT) / eps * gdr_inner_dev(2.0 * gamma * eps, peak, ec, w, lo, hi);
  };
  const double ya = log(e_lo), yb = log(e_hi), ys = log(hi / (2.0 * gamma));
  const double I = (ys > ya && ys < yb) ? gl_composite(gl, g, ya, ys) + gl_composite(gl, g, ys, yb)
                                        : gl_composite(gl, g, ya, yb);
  return I / (2.0 * gamma * gamma);
}

__global__ void k_tables(crp_tables_desc d, const GLRule gl, double* beta, double* pion,
                         double* gdr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const double l0 = log(d.gamma_lo), l1 = log(d.gamma_hi);
  const double gamma = exp(l0 + (l1 - l0) * (double)i / (double)(d.n - 1));
  const double kT = kBoltz * d.T_cmb;
  const double mb = 1.0e-31;
  double b = beta_pair_dev(gl, gamma, kT);
  for (int k = 0; k < 2; ++k)  // synthetic infrared / optical components
    if (d.irb_dilution[k] > 0.0)
      b = b + d.irb_dilution[k] * beta_pair_dev(gl, gamma, kBoltz * d.irb_T_K[k]);
  beta[i] = b * d.length_unit_m;
  pion[i] = rate_pion_dev(gamma, kT, d.pion_sigma_mb * mb, d.pion_eth_eV) * d.length_unit_m;
  gdr[i] = rate_gdr_dev(gl, gamma, kT, d.gdr_peak_mb * mb, d.gdr_center_eV, 0.5 * d.gdr_fwhm_eV,
                        d.gdr_lo_eV, d.gdr_hi_eV) * d.length_unit_m;
}

// Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's
// method from the Tricomi-type initial estimate, P_n and P_n' by recurrence.
void legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double pn = 0.0, dpn = 0.0;
    for (int it = 0; it < 64; ++it) {
      double pm1 = 1.0, p = z;
      for (int k = 1; k < n; ++k) {
        const double pp = ((2 * k + 1) * z * p - k * pm1) / (k + 1);
        pm1 = p;
        p = pp;
      }
      pn = p;
      dpn = n * (pm1 - z * p) / (1.0 - z * z);
      const double dz = pn / dpn;
      z -= dz;
      if (fabs(dz) <= 1e-17) break;
    }
    double pm1 = 1.0, p = z;
    for (int k = 1; k < n; ++k) {
      const double pp = ((2 * k + 1) * z * p - k * pm1) / (k + 1);
      pm1 = p;
      p = pp;
    }
    dpn = n * (pm1 - z * p) / (1.0 - z * z);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
}

}  // namespace

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  legendre_rule(n, x, w);
}

crp_status tables_compute(const crp_tables_desc* d, double* beta, double* pion, double* gdr,
                          cudaStream_t s) {
  GLRule gl;
  {
    std::vector<double> x, w;
    legendre_rule(kGL, x, w);
    for (int j = 0; j < kGL; ++j) {
      gl.x[j] = x[j];
      gl.w[j] = w[j];
    }
  }
  const int block = 64;
  const int grid = (int)((d->n + block - 1) / block);
  k_tables<<<grid, block, 0, s>>>(*d, gl, beta, pion, gdr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? CRP_OK : fail_cuda(e, "table kernel");
}

}  // namespace crp
