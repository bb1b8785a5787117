// Device arithmetic for the FPE kernels: power-of-two scaling by exponent-field
// construction, double-double error-free transformations (TwoSum: Knuth,
// TAOCP 4.2.2; TwoProd via FMA), and an extended-exponent complex
// double-double type used for the valuation monomial z^l (§8.2) and for
// combining partial window sums.
#pragma once

#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>
#include <string.h>

#include "fpe_internal.h"

namespace fpe {

// 2^k for k in [-1022, 1023], built from the exponent field (no FP64 op).
__device__ __forceinline__ double pow2i(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// x * 2^k, exact whenever the result is a normal double; saturates to 0 or
// inf beyond the range (one multiply in the common case, at most three).
__device__ __forceinline__ double scale2(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * pow2i(k);
  k = max(-3000, min(3000, k));
  int k1 = k / 3, k2 = (k - k1) / 2, k3 = k - k1 - k2;
  return ((x * pow2i(k1)) * pow2i(k2)) * pow2i(k3);
}

// floor(log2 |x|) + 1 for finite nonzero normal or subnormal x (frexp exponent)
__device__ __forceinline__ int frexp_exp(double x) {
  int hi = __double2hiint(x);
  int ex = (hi >> 20) & 0x7ff;
  if (ex != 0) return ex - 1022;
  int f;
  frexp(x, &f);
  return f;
}

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  return {p, fma(a, b, -p)};
}

// Extended-exponent complex double-double: ((rh + rl) + i (ih + il)) * 2^e,
// kept normalised so that max(|rh|, |ih|) lies in [0.5, 1) or both are zero.
struct xdd {
  double rh, rl, ih, il;
  long long e;
};

__device__ __forceinline__ xdd xdd_zero() { return {0.0, 0.0, 0.0, 0.0, 0}; }

__device__ __forceinline__ xdd xdd_norm(xdd x) {
  double m = fmax(fabs(x.rh), fabs(x.ih));
  if (m == 0.0) {
    // fold low parts (only reachable after exact cancellation of the high parts)
    dd r = fast_two_sum(x.rl, 0.0), i = fast_two_sum(x.il, 0.0);
    x.rh = r.hi;
    x.rl = 0.0;
    x.ih = i.hi;
    x.il = 0.0;
    m = fmax(fabs(x.rh), fabs(x.ih));
    if (m == 0.0) return xdd_zero();
  }
  int f = frexp_exp(m);
  if (f != 0) {
    double s = scale2(1.0, -f);
    if (f >= -1021 && f <= 1022) {
      x.rh *= s;
      x.rl *= s;
      x.ih *= s;
      x.il *= s;
    } else {
      x.rh = scale2(x.rh, -f);
      x.rl = scale2(x.rl, -f);
      x.ih = scale2(x.ih, -f);
      x.il = scale2(x.il, -f);
    }
    x.e += f;
  }
  return x;
}

// From an FP64 complex value times 2^e.
__device__ __forceinline__ xdd xdd_from(double re, double im, long long e) {
  xdd x = {re, 0.0, im, 0.0, e};
  return xdd_norm(x);
}

// x * x
__device__ __forceinline__ xdd xdd_sqr(xdd x) {
  dd p1 = two_prod(x.rh, x.rh), p2 = two_prod(x.ih, x.ih), p3 = two_prod(x.rh, x.ih);
  dd s = two_sum(p1.hi, -p2.hi);
  double t = s.lo + (p1.lo - p2.lo) + 2.0 * (x.rh * x.rl - x.ih * x.il);
  dd re = two_sum(s.hi, t);
  double ti = p3.lo + x.rh * x.il + x.rl * x.ih;
  dd im = fast_two_sum(2.0 * p3.hi, 2.0 * ti);
  xdd r = {re.hi, re.lo, im.hi, im.lo, 2 * x.e};
  return xdd_norm(r);
}

// x * (zr + i zi) with zr, zi plain doubles (scaled by 2^ze)
__device__ __forceinline__ xdd xdd_mul_d(xdd x, double zr, double zi, long long ze) {
  dd p1 = two_prod(x.rh, zr), p2 = two_prod(x.ih, zi);
  dd s = two_sum(p1.hi, -p2.hi);
  double t = s.lo + (p1.lo - p2.lo) + (x.rl * zr - x.il * zi);
  dd re = two_sum(s.hi, t);
  dd p3 = two_prod(x.rh, zi), p4 = two_prod(x.ih, zr);
  dd u = two_sum(p3.hi, p4.hi);
  double ti = u.lo + (p3.lo + p4.lo) + (x.rl * zi + x.il * zr);
  dd im = two_sum(u.hi, ti);
  xdd r = {re.hi, re.lo, im.hi, im.lo, x.e + ze};
  return xdd_norm(r);
}

// x * y
__device__ __forceinline__ xdd xdd_mul(xdd x, xdd y) {
  dd p1 = two_prod(x.rh, y.rh), p2 = two_prod(x.ih, y.ih);
  dd s = two_sum(p1.hi, -p2.hi);
  double t = s.lo + (p1.lo - p2.lo) + (x.rh * y.rl + x.rl * y.rh) - (x.ih * y.il + x.il * y.ih);
  dd re = two_sum(s.hi, t);
  dd p3 = two_prod(x.rh, y.ih), p4 = two_prod(x.ih, y.rh);
  dd u = two_sum(p3.hi, p4.hi);
  double ti = u.lo + (p3.lo + p4.lo) + (x.rh * y.il + x.rl * y.ih) + (x.ih * y.rl + x.il * y.rh);
  dd im = two_sum(u.hi, ti);
  xdd r = {re.hi, re.lo, im.hi, im.lo, x.e + y.e};
  return xdd_norm(r);
}

// x + y (both normalised)
__device__ __forceinline__ xdd xdd_add(xdd x, xdd y) {
  bool xz = (x.rh == 0.0 && x.ih == 0.0), yz = (y.rh == 0.0 && y.ih == 0.0);
  if (yz) return x;
  if (xz) return y;
  if (x.e < y.e) {
    xdd t = x;
    x = y;
    y = t;
  }
  long long sh = y.e - x.e;  // <= 0
  if (sh < -220) return x;   // y below 2^-218 of x: beyond double-double precision
  double s = pow2i((int)sh);
  dd re = two_sum(x.rh, y.rh * s), im = two_sum(x.ih, y.ih * s);
  re.lo += x.rl + y.rl * s;
  im.lo += x.il + y.il * s;
  dd r2 = two_sum(re.hi, re.lo), i2 = two_sum(im.hi, im.lo);
  xdd r = {r2.hi, r2.lo, i2.hi, i2.lo, x.e};
  return xdd_norm(r);
}

// (zr + i zi)^n for n >= 0, left-to-right binary powering (§8.2: z^l by
// repeated squaring, at most 2 log2 l products), in extended double-double.
__device__ __forceinline__ xdd xdd_pow(double zr, double zi, long long n) {
  if (n <= 0) return {0.5, 0.0, 0.0, 0.0, 1};
  // split z = m 2^f with max(|m|) in [0.5, 1) so that the running power stays normalised
  int f = frexp_exp(fmax(fabs(zr), fabs(zi)));
  double mr = scale2(zr, -f), mi = scale2(zi, -f);
  xdd r = xdd_from(mr, mi, 0);
  int top = 63 - __clzll(n);
  for (int b = top - 1; b >= 0; --b) {
    r = xdd_sqr(r);
    if ((n >> b) & 1) r = xdd_mul_d(r, mr, mi, 0);
  }
  r.e += (long long)f * n;
  return r;
}

// One Horner step h <- h w + b on complex (or real, CZ/CC false) values.
// COMP: compensated step -- the rounding errors of the products and sums are
// recovered exactly by TwoProd and TwoSum and accumulated by a second
// recurrence c <- c w + (errors); the value is h + c.  The compensated Horner
// schemes cited in §1 bound the error by u|P| + gamma_2n^2 sum |a_k||z|^k.
template <bool CC, bool CZ, bool COMP>
__device__ __forceinline__ void horner_step(double &hr, double &hm, double &cr, double &cm, double wr, double wi,
                                            double br, double bi) {
  if (!COMP) {
    if (CZ) {
      double nr = fma(hr, wr, fma(-hm, wi, br));
      double ni = fma(hr, wi, fma(hm, wr, bi));
      hr = nr;
      hm = ni;
    } else {
      hr = fma(hr, wr, br);
      if (CC) hm = fma(hm, wr, bi);
    }
  } else if (CZ) {
    dd p1 = two_prod(hr, wr), p2 = two_prod(hm, wi), p3 = two_prod(hr, wi), p4 = two_prod(hm, wr);
    dd s1 = two_sum(p1.hi, -p2.hi), s2 = two_sum(s1.hi, br);
    dd t1 = two_sum(p3.hi, p4.hi), t2 = two_sum(t1.hi, bi);
    double er = ((p1.lo - p2.lo) + s1.lo) + s2.lo;
    double ei = ((p3.lo + p4.lo) + t1.lo) + t2.lo;
    double ncr = fma(cr, wr, fma(-cm, wi, er));
    double nci = fma(cr, wi, fma(cm, wr, ei));
    cr = ncr;
    cm = nci;
    hr = s2.hi;
    hm = t2.hi;
  } else {
    dd p1 = two_prod(hr, wr), s2 = two_sum(p1.hi, br);
    cr = fma(cr, wr, p1.lo + s2.lo);
    hr = s2.hi;
    if (CC) {
      dd q1 = two_prod(hm, wr), t2 = two_sum(q1.hi, bi);
      cm = fma(cm, wr, q1.lo + t2.lo);
      hm = t2.hi;
    }
  }
}

// 1/m in double-double for a complex m with max(|mr|, |mi|) in [0.5, 1):
// conj(m) / |m|^2, |m|^2 summed exactly from TwoProd terms, each quotient
// refined by one FMA-based correction step.
struct cdd {
  double rh, rl, ih, il;
};
__device__ __forceinline__ dd dd_div_d(double a, dd b) {
  double q1 = a / b.hi;
  double r = fma(-q1, b.hi, a) - q1 * b.lo;
  double q2 = r / b.hi;
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ cdd recip_dd(double mr, double mi) {
  dd p1 = two_prod(mr, mr), p2 = two_prod(mi, mi);
  dd s = two_sum(p1.hi, p2.hi);
  dd n2 = fast_two_sum(s.hi, s.lo + p1.lo + p2.lo);
  dd ur = dd_div_d(mr, n2), ui = dd_div_d(-mi, n2);
  return {ur.hi, ur.lo, ui.hi, ui.lo};
}

// ---------------------------------------------------------------------------
// z^n on the integer pipe.  On this GPU a 64-bit integer multiply-high issues
// about four times as fast as an FP64 FMA and 32-bit multiply-adds about 37
// times, so the valuation power (§8.2: z^l by repeated squaring) is computed
// in 128-bit fixed-point mantissas: a value is ((-1)^sx X + i (-1)^sy Y) 2^(e-126)
// with X, Y unsigned 128-bit and max(X, Y) in [2^126, 2^127).  Each product
// keeps the top 128 bits of the 256-bit product (truncation error below 2^-123
// relative), so after the at most 62 squarings and products of a 31-bit
// exponent the relative error stays below 2^-85, far inside double-double use.
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

struct xint {
  u128 x, y;
  int sx, sy;  // signs (1 = negative)
  long long e;
};

__host__ __device__ __forceinline__ unsigned long long umulhi64(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((u128)a * b) >> 64);
#endif
}

// top 128 bits of the 256-bit product a b (the two lowest partial products dropped)
__host__ __device__ __forceinline__ u128 mulhi128(u128 a, u128 b) {
  const unsigned long long a1 = (unsigned long long)(a >> 64), a0 = (unsigned long long)a;
  const unsigned long long b1 = (unsigned long long)(b >> 64), b0 = (unsigned long long)b;
  u128 p = (u128)a1 * b1;
  p += umulhi64(a1, b0);
  p += umulhi64(a0, b1);
  return p;
}

__host__ __device__ __forceinline__ int clz128(u128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
#ifdef __CUDA_ARCH__
  return hi ? __clzll(hi) : 64 + __clzll(lo);
#else
  return hi ? __builtin_clzll(hi) : (lo ? 64 + __builtin_clzll(lo) : 128);
#endif
}

// signed magnitude addition (a, sa) + (b, sb)
__host__ __device__ __forceinline__ void sadd128(u128 a, int sa, u128 b, int sb, u128 &r, int &sr) {
  if (sa == sb) {
    r = a + b;
    sr = sa;
  } else if (a >= b) {
    r = a - b;
    sr = sa;
  } else {
    r = b - a;
    sr = sb;
  }
}

__host__ __device__ __forceinline__ xint xint_norm(u128 x, int sx, u128 y, int sy, long long e) {
  const u128 m = x > y ? x : y;
  xint r;
  if (m == 0) {
    r.x = r.y = 0;
    r.sx = r.sy = 0;
    r.e = 0;
    return r;
  }
  const int sh = clz128(m) - 1;  // bring the top bit to position 126
  if (sh > 0) {
    x <<= sh;
    y <<= sh;
  } else if (sh < 0) {
    x >>= 1;
    y >>= 1;
  }
  r.x = x;
  r.y = y;
  r.sx = x ? sx : 0;
  r.sy = y ? sy : 0;
  r.e = e - sh;
  return r;
}

__host__ __device__ __forceinline__ unsigned long long dbl_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

// a normalised double component (|c| < 1) as a 128-bit magnitude at scale 2^127
__host__ __device__ __forceinline__ u128 u128_from_unit(double c) {
  const unsigned long long bits = dbl_bits(c) & 0x7fffffffffffffffull;
  const int ex = (int)(bits >> 52);
  if (ex == 0) return 0;  // zero or below 2^-1022: negligible against the unit-size component
  const unsigned long long m = (bits & 0xfffffffffffffull) | 0x10000000000000ull;
  const int sh = ex - 948;  // |c| = m 2^(ex - 1075), scaled by 2^127
  if (sh >= 0) return (u128)m << sh;
  if (sh <= -64) return 0;
  return (u128)(m >> (-sh));
}

__host__ __device__ __forceinline__ xint xint_mul(const xint &a, const xint &b) {
  u128 p1 = mulhi128(a.x, b.x), p2 = mulhi128(a.y, b.y), p3 = mulhi128(a.x, b.y), p4 = mulhi128(a.y, b.x);
  u128 re, im;
  int sre, sim;
  sadd128(p1, a.sx ^ b.sx, p2, 1 ^ a.sy ^ b.sy, re, sre);
  sadd128(p3, a.sx ^ b.sy, p4, a.sy ^ b.sx, im, sim);
  return xint_norm(re, sre, im, sim, a.e + b.e + 2);
}

__host__ __device__ __forceinline__ xint xint_sqr(const xint &a) {
  u128 p1 = mulhi128(a.x, a.x), p2 = mulhi128(a.y, a.y), p3 = mulhi128(a.x, a.y);
  u128 re;
  int sre;
  sadd128(p1, 0, p2, 1, re, sre);
  return xint_norm(re, sre, p3 << 1, a.sx ^ a.sy, 2 * a.e + 2);
}

// (mr + i mi)^n for a unit-size complex (max(|mr|, |mi|) in [0.5, 1)), n >= 1
__host__ __device__ __forceinline__ xint xint_pow_unit(double mr, double mi, long long n) {
  xint z = xint_norm(u128_from_unit(mr), mr < 0.0, u128_from_unit(mi), mi < 0.0, -1);
  xint r = z;
#ifdef __CUDA_ARCH__
  const int top = 63 - __clzll(n);
#else
  const int top = 63 - __builtin_clzll((unsigned long long)n);
#endif
  for (int b = top - 1; b >= 0; --b) {
    r = xint_sqr(r);
    if ((n >> b) & 1) r = xint_mul(r, z);
  }
  return r;
}

// the low 74 bits of a 128-bit magnitude, as a double scaled by 2^-74
__host__ __device__ __forceinline__ double low74_scaled(u128 x) {
  const unsigned long long lo = (unsigned long long)x, up = (unsigned long long)(x >> 64) & 0x3ffull;
  return (double)up * 0x1p-10 + (double)lo * 0x1p-74;
}

// extended double-double from a 128-bit mantissa pair
__device__ __forceinline__ xdd xdd_from_xint(const xint &v) {
  // component = (-1)^s (H + L 2^-74) 2^(e - 52), H = X >> 74 (53 bits), L = X mod 2^74
  const double hx = (double)(unsigned long long)(v.x >> 74);
  const double lx = low74_scaled(v.x);
  const double hy = (double)(unsigned long long)(v.y >> 74);
  const double ly = low74_scaled(v.y);
  xdd x;
  x.rh = (v.sx ? -hx : hx) * 0x1p-53;
  x.rl = (v.sx ? -lx : lx) * 0x1p-53;
  x.ih = (v.sy ? -hy : hy) * 0x1p-53;
  x.il = (v.sy ? -ly : ly) * 0x1p-53;
  x.e = v.e + 1;
  return xdd_norm(x);
}

// z^n (n >= 0) as extended double-double, computed on the integer pipe.
__device__ __forceinline__ xdd xdd_pow_int(double zr, double zi, long long n) {
  if (n <= 0) return {0.5, 0.0, 0.0, 0.0, 1};
  const int f = frexp_exp(fmax(fabs(zr), fabs(zi)));
  xint r = xint_pow_unit(scale2(zr, -f), scale2(zi, -f), n);
  xdd x = xdd_from_xint(r);
  x.e += (long long)f * n;
  return x;
}

// ---------------------------------------------------------------------------
// Horner steps on the integer pipe.  A partial sum is a complex fixed-point
// value (xr + i xi) 2^G with xr, xi two's-complement 128-bit integers; after
// isum_normalise the larger magnitude has its top bit at position 121.  A
// step h <- h w + b truncates at the frame's unit: 2^-121 of the partial sum
// after a normalisation and at most 16 bits more before the next one (a
// product can lose 2 bits of magnitude, and normalising happens every 8
// steps), so a window of L terms summed top-down has an error of order
// L 2^-104 times the sum of the term magnitudes: the summation order no
// longer matters.  The multiplier w = 2^beta z is used exactly: each
// component is its 53-bit mantissa as a signed 63-bit word; when the two
// exponents are within 10 of each other (more for subnormals) both words
// share one exponent exactly, otherwise each keeps its own and the smaller
// product is shifted into the larger's frame (the SPLIT form).  G
// is a 64-bit exponent, so nothing overflows.
//
// Magnitude budget: a product (x w) >> 64 with |w| < 2^63 has at most half
// the magnitude of x, so each component of h w is at most max(|xr|, |xi|),
// and a coefficient adds less than 2^121 (larger ones move the frame up).
// From < 2^122 after normalising, eight steps stay below 2^125 (mulhi_s
// needs < 2^127): callers normalise at least every eight steps.  No FP64
// instruction is used.
// ---------------------------------------------------------------------------
typedef __int128 i128;

constexpr int kIsumTop = 121;        // top bit after normalising
constexpr int kIsumMaxSteps = 8;     // steps between normalisations
constexpr int kIsumCoefShift = 68;   // a coefficient 53-bit mantissa sits at most this far up

struct isum {
  i128 xr, xi;
  long long G;
};

// frame of a zero sum: far below any coefficient, so the next nonzero
// coefficient sets the frame (and steps of a zero sum cannot overflow G)
constexpr long long kIsumZeroFrame = -(1LL << 60);

// w = wr 2^(E - dr) + i wi 2^(E - di), |wr|, |wi| < 2^63; split == 0 means
// dr == di == 0 (one shared exponent)
struct iw {
  long long wr, wi;
  int dr, di, split;
  long long E;
};

// x = (-1)^s m 2^e with m < 2^53 (m = 0 for x = 0)
__host__ __device__ __forceinline__ void decode_dbl(double x, unsigned long long &m, int &e, int &s) {
  const unsigned long long bits = dbl_bits(x);
  s = (int)(bits >> 63);
  const int ex = (int)((bits >> 52) & 0x7ff);
  m = bits & 0xfffffffffffffull;
  if (ex == 0) {
    e = -1074;
  } else {
    m |= 0x10000000000000ull;
    e = ex - 1075;
  }
}

__host__ __device__ __forceinline__ int bitlen64(unsigned long long m) {
#ifdef __CUDA_ARCH__
  return m ? 64 - __clzll(m) : 0;
#else
  return m ? 64 - __builtin_clzll(m) : 0;
#endif
}

__host__ __device__ __forceinline__ iw iw_from(double zr, double zi) {
  unsigned long long mr, mi;
  int er, ei, sr, si;
  decode_dbl(zr, mr, er, sr);
  decode_dbl(zi, mi, ei, si);
  iw w;
  // each mantissa with its top bit at 62, exponents Er, Ei of the word's unit
  const int shr = mr ? 63 - bitlen64(mr) : 0, shi = mi ? 63 - bitlen64(mi) : 0;
  const long long Er = (long long)er - shr, Ei = (long long)ei - shi;
  w.E = mr ? (mi ? (Er > Ei ? Er : Ei) : Er) : Ei;
  long long dr = mr ? w.E - Er : 0, di = mi ? w.E - Ei : 0;
  // when the smaller word has at least that many trailing zeros (10 for a
  // normal double) it moves down to the larger's unit exactly: one exponent
  const int sdr = (dr > 0 && dr <= shr) ? (int)dr : 0;
  const int sdi = (di > 0 && di <= shi) ? (int)di : 0;
  const unsigned long long ur = (mr << shr) >> sdr, ui = (mi << shi) >> sdi;
  dr -= sdr;
  di -= sdi;
  w.wr = sr ? -(long long)ur : (long long)ur;
  w.wi = si ? -(long long)ui : (long long)ui;
  w.dr = (int)(dr < 127 ? dr : 127);
  w.di = (int)(di < 127 ? di : 127);
  w.split = (w.dr | w.di) != 0;
  return w;
}

// (x w) / 2^64 for |x| < 2^127, |w| < 2^63, within 1 of the exact quotient
// (the low partial product is truncated)
__host__ __device__ __forceinline__ i128 mulhi_s(i128 x, long long w) {
  const long long x1 = (long long)(x >> 64);
  const unsigned long long x0 = (unsigned long long)x;
  const unsigned long long h0 = umulhi64(x0, (unsigned long long)w) - (w < 0 ? x0 : 0ull);
  return (i128)x1 * w + (i128)(long long)h0;
}

// (-1)^s m 2^sh as a signed 128-bit value, sh <= kIsumCoefShift (truncated below 2^0)
__host__ __device__ __forceinline__ i128 place53(unsigned long long m, int s, long long sh) {
  const long long v = s ? -(long long)m : (long long)m;
  if (sh >= 0) return (i128)((u128)(i128)v << sh);
  return sh > -64 ? (i128)(v >> (-sh)) : (i128)(v >> 63);
}

__host__ __device__ __forceinline__ void isum_normalise(isum &h) {
  const u128 m = (u128)(h.xr ^ (h.xr >> 127)) | (u128)(h.xi ^ (h.xi >> 127));
  if (!m) {  // 0 or -1 (below the frame's unit): a zero sum
    h.xr = h.xi = 0;
    h.G = kIsumZeroFrame;
    return;
  }
  const int d = clz128(m) - (127 - kIsumTop);
  if (d > 0) {
    h.xr = (i128)((u128)h.xr << d);
    h.xi = (i128)((u128)h.xi << d);
  } else if (d < 0) {
    h.xr >>= -d;
    h.xi >>= -d;
  }
  h.G -= d;
}

// fixed-point copy of the complex double hr + i hm, normalised (exact unless
// the two parts are more than 68 binary orders apart)
__host__ __device__ __forceinline__ isum isum_from(double hr, double hm) {
  unsigned long long mr, mi;
  int er, ei, sr, si;
  decode_dbl(hr, mr, er, sr);
  decode_dbl(hm, mi, ei, si);
  isum h;
  if (!mr && !mi) {
    h.xr = h.xi = 0;
    h.G = kIsumZeroFrame;
    return h;
  }
  const long long tr = mr ? (long long)er + bitlen64(mr) - 1 : LLONG_MIN;
  const long long ti = mi ? (long long)ei + bitlen64(mi) - 1 : LLONG_MIN;
  h.G = (tr > ti ? tr : ti) - kIsumTop;
  h.xr = mr ? place53(mr, sr, er - h.G) : (i128)0;
  h.xi = mi ? place53(mi, si, ei - h.G) : (i128)0;
  return h;
}

// h <- h w 2^shift + (br + i bi) without normalising; CZ: complex w, CC:
// complex coefficient (h is complex when either is), SPLIT: w with two
// exponents.  we64 = w.E + shift + 64.
template <bool CC, bool CZ, bool SPLIT>
__host__ __device__ __forceinline__ void isum_step(isum &h, const iw &w, long long we64, double br, double bi) {
  constexpr bool CH = CC || CZ;
  i128 re, im = 0;
  if (CZ) {
    if (SPLIT) {
      re = (mulhi_s(h.xr, w.wr) >> w.dr) - (mulhi_s(h.xi, w.wi) >> w.di);
      im = (mulhi_s(h.xr, w.wi) >> w.di) + (mulhi_s(h.xi, w.wr) >> w.dr);
    } else {
      re = mulhi_s(h.xr, w.wr) - mulhi_s(h.xi, w.wi);
      im = mulhi_s(h.xr, w.wi) + mulhi_s(h.xi, w.wr);
    }
  } else {
    re = mulhi_s(h.xr, w.wr);
    if (CH) im = mulhi_s(h.xi, w.wr);
  }
  long long G = h.G + we64;
  unsigned long long mr, mi = 0;
  int er, ei = 0, s_r, s_i = 0;
  decode_dbl(br, mr, er, s_r);
  if (CC) decode_dbl(bi, mi, ei, s_i);
  // a coefficient of 2^121 or more in this frame moves the frame up first
  long long need = G;
  if (mr && (long long)er - need > kIsumCoefShift) need = (long long)er - kIsumCoefShift;
  if (CC && mi && (long long)ei - need > kIsumCoefShift) need = (long long)ei - kIsumCoefShift;
  if (need > G) {
    const int d = (int)(need - G < 127 ? need - G : 127);
    re >>= d;
    im >>= d;
    G = need;
  }
  if (mr) re += place53(mr, s_r, (long long)er - G);
  if (CC && mi) im += place53(mi, s_i, (long long)ei - G);
  h.xr = re;
  h.xi = im;
  h.G = G;
}

// extended double-double of a fixed-point sum
__device__ __forceinline__ xdd xdd_from_isum(const isum &h) {
  const int sr = h.xr < 0, si = h.xi < 0;
  const u128 ar = sr ? (u128)(-h.xr) : (u128)h.xr, ai = si ? (u128)(-h.xi) : (u128)h.xi;
  if (!ar && !ai) return xdd_zero();
  return xdd_from_xint(xint_norm(ar, sr, ai, si, h.G + 126));
}

// Normalised FP64 output (fpe_xc64) from an extended double-double value.
__device__ __forceinline__ fpe_xc64 xdd_out(xdd x) {
  double re = x.rh + x.rl, im = x.ih + x.il;
  double m = fmax(fabs(re), fabs(im));
  fpe_xc64 o;
  if (m == 0.0) {
    o.re = 0.0;
    o.im = 0.0;
    o.e = 0;
    return o;
  }
  int f = frexp_exp(m);
  o.re = scale2(re, -f);
  o.im = scale2(im, -f);
  o.e = x.e + f;
  return o;
}

}  // namespace fpe
