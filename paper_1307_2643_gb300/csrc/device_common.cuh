// device_common.cuh -- device primitives: counter-based random numbers,
// lineage ids and the Cash-Karp tableau.
#pragma once

#include <stdint.h>
#include <string.h>

namespace crp {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): per round, two 32x32 -> 64-bit products of
// counter words 0 and 2 with 0xD2511F53 / 0xCD9E8D57; the new counter is
// (hi(c2 m1) ^ c1 ^ k0, lo(c2 m1), hi(c0 m0) ^ c3 ^ k1, lo(c0 m0)); the key
// advances by the Weyl increments 0x9E3779B9 / 0xBB67AE85 between rounds.
struct Philox4 {
  uint32_t v0, v1, v2, v3;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each 32 x 32 -> 64-bit product in one wide multiply
    const uint32_t hi_a = mulhi32(0xD2511F53u, c0);
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t hi_b = mulhi32(0xCD9E8D57u, c2);
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi_b ^ c1 ^ k0;
    const uint32_t n2 = hi_a ^ c3 ^ k1;
    c0 = n0;
    c1 = lo_b;
    c2 = n2;
    c3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Philox4{c0, c1, c2, c3};
}

// Open-interval uniform from two words: (top 52 bits of hi:lo + 1/2) * 2^-52.
__host__ __device__ __forceinline__ double u01_open(uint32_t lo, uint32_t hi) {
  const unsigned long long v = ((unsigned long long)hi << 32) | lo;
  return ((double)(v >> 12) + 0.5) * 2.220446049250313080847263336181640625e-16;
}

// Stream tags of the counter (draw, tag, id_lo, id_hi).
constexpr uint32_t TAG_FIELD = 1;
constexpr uint32_t TAG_INTERACTION = 2;
constexpr uint32_t TAG_COSMOLOGY = 5;  // a-posteriori correction: product pick

__host__ __device__ __forceinline__ Philox4 draw4(uint64_t seed, uint32_t tag, uint64_t id,
                                                  uint32_t draw) {
  return philox4x32_10(draw, tag, (uint32_t)id, (uint32_t)(id >> 32), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) over a Weyl step:
// id of the secondary of a parent's event number `ev`.
__host__ __device__ __forceinline__ uint64_t lineage_id(uint64_t parent, uint32_t ev) {
  uint64_t z = parent + 0x9E3779B97F4A7C15ull * ((uint64_t)ev + 1ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Cash-Karp 5(4) (Cash & Karp, ACM TOMS 16, 201, 1990): stage coefficients,
// fifth-order weights and (fifth - embedded fourth) weights, each the
// nearest double of its rational.
namespace ck {
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 3.0 / 10.0, a42 = -9.0 / 10.0, a43 = 6.0 / 5.0;
constexpr double a51 = -11.0 / 54.0, a52 = 5.0 / 2.0, a53 = -70.0 / 27.0, a54 = 35.0 / 27.0;
constexpr double a61 = 1631.0 / 55296.0, a62 = 175.0 / 512.0, a63 = 575.0 / 13824.0,
                 a64 = 44275.0 / 110592.0, a65 = 253.0 / 4096.0;
constexpr double w1 = 37.0 / 378.0, w3 = 250.0 / 621.0, w4 = 125.0 / 594.0, w6 = 512.0 / 1771.0;
constexpr double d1 = -277.0 / 64512.0, d3 = 6925.0 / 370944.0, d4 = -6925.0 / 202752.0,
                 d5 = -277.0 / 14336.0, d6 = 277.0 / 7084.0;
}  // namespace ck

// Natural logarithm for the quantities that steer the propagation (free
// paths -ln(u), ln(Gamma) of table lookups): x = 2^k m with m in
// [sqrt(1/2), sqrt(2)], s = (m-1)/(m+1), ln m = 2 atanh(s) summed as the
// series 2 s (1 + s^2/3 + ... + s^26/27) by Horner, ln x = k ln2 + ln m.
// Positive normal finite x only.  Written out operation by operation so that
// a translation unit built without multiply-add contraction reproduces the
// same bits as any other IEEE binary64 evaluation of the same sequence.
__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

__host__ __device__ __forceinline__ double dfrombits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof(x));
  return x;
#endif
}

__host__ __device__ __forceinline__ double series_log(double x) {
  const unsigned long long b = dbits(x);
  int k = (int)((b >> 52) & 0x7ffull) - 1023;
  double m = dfrombits((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
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

// Exponential for the binary64 analytic galactic field, operation by
// operation: x = k ln2 + r (k nearest integer, ln2 split Cody-Waite style
// into a 32-bit high part and a low part), e^r by its Taylor series to
// r^13/13! (Horner), 2^k built in the exponent field.  -700 <= x <= 700.
__device__ __forceinline__ double series_exp(double x) {
  if (x < -700.0) return 0.0;
  const double ln2_hi = 2977044472.0 / 4294967296.0;
  const double ln2_lo = -4.2009150726810847e-11;
  const double kd = floor(x * 1.4426950408889634074 + 0.5);
  const double r = (x - kd * ln2_hi) - kd * ln2_lo;
  double poly = 1.0 / 6227020800.0;
  poly = poly * r + 1.0 / 479001600.0;
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
  const int k = (int)kd;
  const double scale = __longlong_as_double((long long)((unsigned long long)(k + 1023) << 52));
  return poly * scale;
}

// Arctangent of y/x in (-pi, pi], step by step so that the binary64
// multi-arm galactic field is reproducible: t = min(|x|,|y|) / max(|x|,|y|);
// three halvings atan t = 2 atan(t / (1 + sqrt(1 + t^2))) leave t below
// tan(pi/32) < 0.0985, where the Taylor series t - t^3/3 + ... - t^15/15
// (Horner in t^2) has a tail below 1e-17 t; octant and quadrant by
// atan(1/t) = pi/2 - atan t and atan2(y, -x) = pi - atan2(y, x);
// atan2(0, 0) = 0.  Division and square root are the IEEE-rounded ones.
__device__ __forceinline__ double series_atan2(double y, double x) {
  const double ax = fabs(x), ay = fabs(y);
  if (ax == 0.0 && ay == 0.0) return 0.0;
  const bool steep = ay > ax;
  double t = steep ? ax / ay : ay / ax;
#pragma unroll
  for (int i = 0; i < 3; ++i) t = t / (1.0 + sqrt(1.0 + t * t));
  const double t2 = t * t;
  double poly = -1.0 / 15.0;
  poly = poly * t2 + 1.0 / 13.0;
  poly = poly * t2 - 1.0 / 11.0;
  poly = poly * t2 + 1.0 / 9.0;
  poly = poly * t2 - 1.0 / 7.0;
  poly = poly * t2 + 1.0 / 5.0;
  poly = poly * t2 - 1.0 / 3.0;
  poly = poly * t2 + 1.0;
  const double pi = 3.14159265358979323846;
  double a = 8.0 * (t * poly);
  if (steep) a = 0.5 * pi - a;
  if (x < 0.0) a = pi - a;
  return y < 0.0 ? -a : a;
}

// HEALPix RING pixel of a direction (Gorski et al., ApJ 622, 759, 2005):
// 12 nside^2 equal-area pixels; polar caps |z| > 2/3 and the equatorial
// belt, pixels numbered ring by ring from the north pole.
__device__ __forceinline__ int64_t healpix_ring_pixel(int64_t nside, double ux, double uy,
                                                      double uz) {
  const double halfpi = 1.57079632679489661923;
  double phi = atan2(uy, ux);
  if (phi < 0.0) phi += 2.0 * 3.14159265358979323846;
  const double tt = phi / halfpi;  // [0, 4)
  const double za = fabs(uz);
  const int64_t ncap = 2 * nside * (nside - 1);
  const int64_t npix = 12 * nside * nside;
  if (za <= 2.0 / 3.0) {
    const double t1 = (double)nside * (0.5 + tt);
    const double t2 = (double)nside * uz * 0.75;
    const int64_t jp = (int64_t)floor(t1 - t2);
    const int64_t jm = (int64_t)floor(t1 + t2);
    const int64_t ir = nside + 1 + jp - jm;
    const int64_t kshift = 1 - (ir & 1);
    int64_t ip = (jp + jm - nside + kshift + 1) / 2;
    ip = ((ip % (4 * nside)) + 4 * nside) % (4 * nside);
    return ncap + (ir - 1) * 4 * nside + ip;
  }
  const double tp = tt - floor(tt);
  const double tmp = (double)nside * sqrt(3.0 * (1.0 - za));
  const int64_t jp = (int64_t)floor(tp * tmp);
  const int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
  const int64_t ir = jp + jm + 1;
  int64_t ip = (int64_t)floor(tt * (double)ir);
  ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
  if (uz > 0.0) return 2 * ir * (ir - 1) + ip;
  return npix - 2 * ir * (ir + 1) + ip;
}

// floor(a) of a binary32 value a within `guard` of the exact value it
// stands for: true when no integer lies within `guard` of a, so that the
// exact value has the same floor (false for NaN, infinities and |a| >= 2^23,
// where a - floor(a) is 0).  32-bit conversion: |a| < 2^23 when true.
__device__ __forceinline__ bool floor_sure(float a, float guard, int* out) {
  const float fl = floorf(a);
  const float f = a - fl;  // exact for |a| < 2^23
  *out = (int)fl;
  return f >= guard && f <= 1.f - guard;
}

// binary32 value of a binary64 x with the significand truncated to 24 bits
// (relative error below 2^-23), by integer operations on its bits: +-0 below
// the normal binary32 range, +-infinity above it, NaN for NaN.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) {
    const bool nan = e == 2047 - 1023 + 127 && (((hi & 0xfffffu) | lo) != 0u);
    return __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
  }
  return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// f32_trunc for |x| < 2 (direction components) in fewer operations: for a
// binary64 exponent field e in [897, 1023] (2^-126 <= |x| < 2) the field's
// top two bits are 01, so shifting the upper word left by three (with the
// lower word's top three bits shifted in) leaves e - 512 above the 23
// significand bits, and subtracting 384 there rebiases it to e - 896.  Below
// that range the result is +-0; from 2 on, f32_trunc itself.
__device__ __forceinline__ float f32_trunc_unit(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned ah = hi & 0x7fffffffu, sign = hi & 0x80000000u;
  if (ah >= 0x40000000u) return f32_trunc(x);
  const unsigned m = __funnelshift_l(lo, hi, 3) - (384u << 23);
  return __uint_as_float(ah < (897u << 20) ? sign : (sign | m));
}

// 1 - |z| for 1/2 <= |z| <= 1 (exact in binary64: the integer
// 2^52 - significand bits, times 2^-53), rounded to binary32 from its two
// 32-bit halves (relative error below 2^-23).
__device__ __forceinline__ float one_minus_abs_f32(double z) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(z) & 0x7fffffffffffffffull;
  if (b >= 0x3ff0000000000000ull) return 0.f;  // |z| = 1
  const unsigned long long d = (1ull << 52) - (b & 0x000fffffffffffffull);
  const float v = (float)(unsigned)(d >> 32) * 4294967296.f + (float)(unsigned)d;
  return v * 1.1102230246251565404e-16f;  // 2^-53
}

// The phase t = phi / (pi/2) in [0, 4) of phi = atan2(y, x) mod 2 pi, in
// binary32 without atan2f or a division by pi/2.  The first-octant part is
// g = (2/pi) atan(r), r = min(|x|, |y|) / max(|x|, |y|) in [0, 1], as r P(r^2)
// with P of degree 7: a least-squares fit of (2/pi) atan(r) / r on Chebyshev
// nodes in r^2, reweighted (Lawson's iteration) towards the minimax error
// of r P(r^2).  Its coefficients, rounded to binary32, are within 4.5e-8 of
// (2/pi) atan(r) on [0, 1] in exact arithmetic; the binary32 Horner steps
// add at most 1.5e-7 (each fma rounds by 2^-24 of a partial sum below 0.64,
// the partial sums' errors shrink by r^2 <= 1).  The octant and quadrant
// then give t = off + sgn g in one fma (half an ulp below 4: 1.2e-7), and
// the quotient r by __fdividef (2 ulp) moves g by at most 7.6e-8.  In all,
// |t - exact| < 3.9e-7 for binary32 x and y (none is subnormal: f32_trunc
// flushes those to zero).  Both zero gives t = 0, as atan2(0, 0) = 0.
__device__ __forceinline__ float phase_quarter_turns(float x, float y) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mn = fminf(ax, ay), mx = fmaxf(ax, ay);
  const float r = mx > 0.f ? __fdividef(mn, mx) : 0.f;
  const float s = r * r;
  float p = -0.002581184497103095f;
  p = fmaf(p, s, 0.01391826756298542f);
  p = fmaf(p, s, -0.03559470921754837f);
  p = fmaf(p, s, 0.06138399615883827f);
  p = fmaf(p, s, -0.08854503184556961f);
  p = fmaf(p, s, 0.12698377668857574f);
  p = fmaf(p, s, -0.21218448877334595f);
  p = fmaf(p, s, 0.6366193294525146f);
  const float g = p * r;
  // quadrant (x >= 0, y >= 0): a; (x < 0, y >= 0): 2 - a; (x < 0, y < 0):
  // 2 + a; (x >= 0, y < 0): 4 - a; with a = g, or 1 - g above the diagonal
  const bool west = x < 0.f, south = y < 0.f;
  const float base = west ? 2.f : (south ? 4.f : 0.f);
  const float sg = west == south ? 1.f : -1.f;
  const bool steep = ay > ax;
  return fmaf(steep ? -sg : sg, g, steep ? base + sg : base);
}

// The same pixel as healpix_ring_pixel of (ux, uy, uz), or of its opposite
// for NEG, with the floors taken in binary32 and binary64 used only within a
// guard band of a pixel boundary.  Error of every binary32 floor argument
// against its exact value, for nside <= 8192: inputs truncated to binary32
// (2^-23 relative: 7.6e-8 on the phase), the phase itself (3.9e-7, see
// phase_quarter_turns), so t within 4.7e-7.  Equatorial belt: the floor
// arguments nside t + nside (0.5 -+ 0.75 z) are one fma each (one rounding,
// 2^-24 of 5 nside), with nside (0.5 -+ 0.75 z) from z truncated (6e-8
// nside) and two roundings (1.2e-7 nside): < nside * 9.5e-7.  Polar caps:
// t - floor(t) exact, the cap formula's 1 - |z| formed exactly before its
// rounding, the products with nside, sqrt and the ring index: < nside *
// 9e-7.  The guard, nside * 4e-6, is 4.2x the larger (2e-5 for the phase
// itself, 40x); outside it the binary32 floor
// equals the exact floor and so the binary64 one, inside it the binary64
// path decides.  Only 32-bit integer conversions and binary32 arithmetic
// run outside the guard band.
// The binary32 part of healpix_ring_pixel_guarded: true, with the pixel, when
// every floor it takes is outside its guard band (the pixel then equals the
// binary64 one); false when the binary64 computation must decide.
template <bool NEG>
__device__ __forceinline__ bool healpix_ring_pixel_try(int64_t nside, double ux, double uy,
                                                       double uz, int64_t* out) {
  const float sg = NEG ? -1.f : 1.f;
  const float fx = sg * f32_trunc_unit(ux), fy = sg * f32_trunc_unit(uy),
              fz = sg * f32_trunc_unit(uz);
  const int ns_i = (int)nside;
  const float ns = (float)ns_i;
  const float g = 4e-6f * ns;
  const float tt = phase_quarter_turns(fx, fy);
  int itt;
  bool ok = floor_sure(tt, 2e-5f, &itt);
  const float za = fabsf(fz);
  ok = ok && fabsf(za - 2.f / 3.f) > 1e-6f;
  // pixel indices below 12 nside^2 <= 805,306,368 for nside <= 8192: 32-bit
  int pix = 0;
  if (ok) {
    if (za <= 2.f / 3.f) {
      // nside (0.5 + t) -+ 0.75 nside z, each with one rounding of the sum
      const float vm = ns * fmaf(-0.75f, fz, 0.5f), vp = ns * fmaf(0.75f, fz, 0.5f);
      int jp, jm;
      ok = floor_sure(fmaf(ns, tt, vm), g, &jp) & floor_sure(fmaf(ns, tt, vp), g, &jm);
      const int ir = ns_i + 1 + jp - jm;
      const int kshift = 1 - (ir & 1);
      int ip = (jp + jm - ns_i + kshift + 1) / 2;
      // jp, jm in [0, 5 nside] put ip in [-nside / 2, 4.5 nside + 1], inside
      // [-M, 2M) for M = 4 nside: one conditional add or subtract is ip mod M
      const int M = 4 * ns_i;
      ip = ip < 0 ? ip + M : (ip >= M ? ip - M : ip);
      pix = 2 * ns_i * (ns_i - 1) + (ir - 1) * 4 * ns_i + ip;
    } else {
      const float tp = tt - (float)itt;
      const float tmp = ns * sqrtf(3.f * one_minus_abs_f32(uz));
      int jp, jm, ip;
      ok = floor_sure(tp * tmp, g, &jp) & floor_sure((1.f - tp) * tmp, g, &jm);
      const int ir = jp + jm + 1;
      ok = ok & floor_sure(tt * (float)ir, g, &ip);
      if (ok) {
        // tt in [0, 4] puts ip in [0, 4 ir]: ip mod 4 ir by one subtraction
        if (ip >= 4 * ir) ip -= 4 * ir;
        if (ip < 0) ip += 4 * ir;
        // the sign of z from its bits: z > +0 exactly when the int64 is > 0
        const bool north = NEG ? __double_as_longlong(uz) < 0 && (__double_as_longlong(uz) << 1) != 0
                               : __double_as_longlong(uz) > 0;
        pix = north ? 2 * ir * (ir - 1) + ip : 12 * ns_i * ns_i - 2 * ir * (ir + 1) + ip;
      }
    }
  }
  *out = pix;
  return ok;
}

// The pixel: the binary32 part's when it is sure, else the binary64 one.
template <bool NEG>
__device__ __forceinline__ int64_t healpix_ring_pixel_guarded(int64_t nside, double ux,
                                                              double uy, double uz) {
  int64_t pix;
  if (healpix_ring_pixel_try<NEG>(nside, ux, uy, uz, &pix)) return pix;
  return NEG ? healpix_ring_pixel(nside, -ux, -uy, -uz) : healpix_ring_pixel(nside, ux, uy, uz);
}

// Spatial key of a grid cell for the work-queue sort: the cell's brick
// (cell >> shift, 32 bricks per axis) in Morton order, 15 bits.
__device__ __forceinline__ uint32_t brick_key(int cx, int cy, int cz, const int shift[3]) {
  const uint32_t bx = (uint32_t)(cx >> shift[0]) & 31u, by = (uint32_t)(cy >> shift[1]) & 31u,
                 bz = (uint32_t)(cz >> shift[2]) & 31u;
  uint32_t key = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
    key |= (((bx >> i) & 1u) << (3 * i)) | (((by >> i) & 1u) << (3 * i + 1)) |
           (((bz >> i) & 1u) << (3 * i + 2));
  return key;
}
constexpr int kSortBins = 1 << 15;

// Rigidity key for the work-queue sort: the top 15 bits of the binary32
// rigidity E/Z (8 exponent + 7 mantissa bits), monotone in E/Z; neutral
// candidates last.  Sorting ascending starts the lowest-rigidity candidates
// (smallest Larmor radius: the most steps) first, so the longest histories
// are not left to run alone at the end.
__host__ __device__ __forceinline__ uint32_t rigidity_key(double E, int Z) {
  if (Z <= 0) return (uint32_t)(kSortBins - 1);
  const float r = (float)(E / (double)Z);
  uint32_t b;
  memcpy(&b, &r, 4);
  return (b >> 16) & (uint32_t)(kSortBins - 1);
}

// Proton rest energy [eV] (CODATA 2018).
constexpr double MP_C2_EV = 938.27208816e6;
constexpr double MN_C2_EV = 939.56542052e6;  // neutron rest energy (CODATA 2018)

}  // namespace crp
