// Device arithmetic for the FPE kernels: power-of-two scaling by exponent-field
// construction, double-double error-free transformations (TwoSum: Knuth,
// TAOCP 4.2.2; TwoProd via FMA), and an extended-exponent complex
// double-double type used for the valuation monomial z^l (§8.2) and for
// combining partial window sums.
#pragma once

#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "fpe_internal.h"

namespace fpe {

// 2^k for k in [-1022, 1023], built from the exponent field (no FP64 op).
__host__ __device__ __forceinline__ double pow2i(int k) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)(k + 1023) << 52);
#else
  const unsigned long long u = (unsigned long long)(k + 1023) << 52;
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}

// x * 2^k, exact whenever the result is a normal double; saturates to 0 or
// inf beyond the range (one multiply in the common case, at most three).
__host__ __device__ __forceinline__ double scale2(double x, int k) {
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

// ---------------------------------------------------------------------------
// Rounding-error certificates of the FP64 window sums (a posteriori, rigorous).
//
// Each FP64 Horner pass with an exact multiplier w runs, beside the value, two
// FP32 recurrences on pipes the FP64-bound loops leave idle:
//   E <- |w| E + sum over the step's rounded results r of 2^e(r)   (rounded up)
//   S <- |w| S + |b_k|                                             (rounded down)
// with e(r) = floor(log2 |r|), both scaled by 2^kMagOff.  A rounding to
// nearest that returns r errs by at most 2^(e(r) - 53), and the errors of
// step k reach the result multiplied by w^(k - lo) exactly, so
//   |computed - exact| <= 2^-53 2^-kMagOff E   and   S <= 2^kMagOff sum |b_k| |w|^(k - lo).
// Magnitudes come from the upper word of a double by integer operations:
// err_mag(r) = 2^(e(r) + kMagOff) with floor 2^-126 (a bound for every
// smaller or zero result) and +inf above the FP32 range; |x| 2^kMagOff <=
// mag_up(x) (mantissa cut to 20 bits plus one unit; 2^-126 below the FP32
// range).  The coefficients' magnitudes come from the host (coef_mag_lo in
// fpe_internal.h, one float per coefficient).  A window
// whose values leave the FP32 window [2^-186, 2^68] fails its certificate
// and is summed again exactly.
// ---------------------------------------------------------------------------
constexpr int kMagBias = (1023 - 127 - kMagOff) << 20;  // double exponent field -> float exponent field

__host__ __device__ __forceinline__ int dbl_hi(double x) {
#ifdef __CUDA_ARCH__
  return __double2hiint(x);
#else
  unsigned long long u;
  memcpy(&u, &x, 8);
  return (int)(u >> 32);
#endif
}
__host__ __device__ __forceinline__ float bits_float(int b) {
#ifdef __CUDA_ARCH__
  return __int_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ float err_mag(double r) {
  const int t = (dbl_hi(r) & 0x7ff00000) - kMagBias;
  return bits_float(min(max(t, 1 << 20), 255 << 20) << 3);
}
// upper bound of |x| 2^kMagOff (mantissa cut to 20 bits plus one unit; floor
// 2^-126, +inf above the FP32 range)
__host__ __device__ __forceinline__ float mag_up(double x) {
  const int t = (dbl_hi(x) & 0x7fffffff) - kMagBias;
  return bits_float((min(max(t, (1 << 20) - 1), (255 << 20) - 1) + 1) << 3);
}
// FP32 operations rounded up / down (device: the rounding-mode instructions;
// host: round to nearest, then one step outward)
#ifdef __CUDA_ARCH__
__device__ __forceinline__ float add_up(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float fma_up(float a, float b, float c) { return __fmaf_ru(a, b, c); }
__device__ __forceinline__ float fma_dn(float a, float b, float c) { return __fmaf_rd(a, b, c); }
__device__ __forceinline__ float mul_up(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float mul_dn(float a, float b) { return __fmul_rd(a, b); }
__device__ __forceinline__ float sqrt_up(float a) { return __fsqrt_ru(a); }
__device__ __forceinline__ float sqrt_dn(float a) { return __fsqrt_rd(a); }
#else
inline float add_up(float a, float b) { return nextafterf(a + b, INFINITY); }
inline float fma_up(float a, float b, float c) { return nextafterf(fmaf(a, b, c), INFINITY); }
inline float fma_dn(float a, float b, float c) { return fmaxf(0.0f, nextafterf(fmaf(a, b, c), -INFINITY)); }
inline float mul_up(float a, float b) { return nextafterf(a * b, INFINITY); }
inline float mul_dn(float a, float b) { return fmaxf(0.0f, nextafterf(a * b, -INFINITY)); }
inline float sqrt_up(float a) { return nextafterf(sqrtf(a), INFINITY); }
inline float sqrt_dn(float a) { return fmaxf(0.0f, nextafterf(sqrtf(a), -INFINITY)); }
#endif

// |x| 2^s as a float rounded up / down, from x's upper word by integer
// operations (no FP64 instruction): mantissa cut to 20 bits (plus one unit
// for the upper bound); below the FP32 range 2^-126 / 0, above it +inf / the
// largest float.
template <int s>
__host__ __device__ __forceinline__ float fabs_up(double x) {
  const int t = (dbl_hi(x) & 0x7fffffff) - ((1023 - 127 - s) << 20);
  return bits_float((min(max(t, (1 << 20) - 1), (255 << 20) - 1) + 1) << 3);
}
template <int s>
__host__ __device__ __forceinline__ float fabs_dn(double x) {
  const int t = (dbl_hi(x) & 0x7fffffff) - ((1023 - 127 - s) << 20);
  return bits_float(min(max(t, 0), (254 << 20) | 0xfffff) << 3);
}

// bounds of |xr + i xi| (no scaling; x a multiplier of moderate size)
__host__ __device__ __forceinline__ float cabs_up(double xr, double xi) {
  const float a = fabs_up<0>(xr), b = fabs_up<0>(xi);
  return sqrt_up(fma_up(a, a, mul_up(b, b)));
}
__host__ __device__ __forceinline__ float cabs_dn(double xr, double xi) {
  const float a = fabs_dn<0>(xr), b = fabs_dn<0>(xi);
  return sqrt_dn(fma_dn(a, a, mul_dn(b, b)));
}
// bounds of |(hr + lr) + i (hi + li)| for a double-double complex multiplier
__host__ __device__ __forceinline__ float cabs_up_dd(double hr, double lr, double hi, double li) {
  const float a = add_up(fabs_up<0>(hr), fabs_up<0>(lr)), b = add_up(fabs_up<0>(hi), fabs_up<0>(li));
  return sqrt_up(fma_up(a, a, mul_up(b, b)));
}
__host__ __device__ __forceinline__ float cabs_dn_dd(double hr, double lr, double hi, double li) {
  const float a = fmaxf(fma_dn(-1.0f, fabs_up<0>(lr), fabs_dn<0>(hr)), 0.0f);
  const float b = fmaxf(fma_dn(-1.0f, fabs_up<0>(li), fabs_dn<0>(hi)), 0.0f);
  return sqrt_dn(fma_dn(a, a, mul_dn(b, b)));
}
// 2^k as a float for |k| <= 126
__host__ __device__ __forceinline__ float pow2f_bits(int k) { return bits_float((k + 127) << 23); }

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

// A complex double-double (rh + rl) + i (ih + il).
struct cdd {
  double rh, rl, ih, il;
};

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

// ---------------------------------------------------------------------------
// Fixed-point helpers for the per-window bookkeeping (exact conversions from
// doubles, addition, the reciprocal 1/m, conversion to the output format):
// they run on the integer pipe, which the FP64-bound window kernels leave
// idle, instead of double-double FP64 chains.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ xint xint_neg(xint a) {
  a.sx = a.x ? a.sx ^ 1 : 0;
  a.sy = a.y ? a.sy ^ 1 : 0;
  return a;
}

// |x| 2^-unit as a 128-bit magnitude (x finite, |x| 2^-unit < 2^127), truncated below 2^0
__host__ __device__ __forceinline__ u128 mag_at(double x, long long unit) {
  const unsigned long long bits = dbl_bits(x) & 0x7fffffffffffffffull;
  const int ex = (int)(bits >> 52);
  if (bits == 0) return 0;
  const unsigned long long m = ex ? ((bits & 0xfffffffffffffull) | 0x10000000000000ull) : (bits & 0xfffffffffffffull);
  const long long sh = (long long)(ex ? ex - 1075 : -1074) - unit;
  if (sh >= 0) return sh < 75 ? (u128)m << sh : (u128)0;
  return sh > -64 ? (u128)(m >> (-sh)) : (u128)0;
}

// top binary exponent of |x| (floor(log2 |x|)), x != 0 finite
__host__ __device__ __forceinline__ long long top_exp(double x) {
  const unsigned long long bits = dbl_bits(x) & 0x7fffffffffffffffull;
  const int ex = (int)(bits >> 52);
  if (ex) return ex - 1023;
  unsigned long long m = bits & 0xfffffffffffffull;
  int b = 0;
  while (m >>= 1) ++b;
  return -1074 + b;
}

// the complex value (rh + rl + i (ih + il)) 2^e as an xint, exactly (the
// low parts at most 2^-50 of the high ones in magnitude, as in double-double)
__host__ __device__ __forceinline__ xint xint_from_dd2(double rh, double rl, double ih, double il, long long e) {
  long long t = LLONG_MIN;
  if (rh != 0.0) t = top_exp(rh);
  if (ih != 0.0 && top_exp(ih) > t) t = top_exp(ih);
  if (t == LLONG_MIN) return xint_norm(0, 0, 0, 0, 0);
  const long long unit = t - 123;  // top bit at 123: room for the low part and a carry
  auto comp = [unit](double h, double l, u128 &m, int &sg) {
    const u128 a = mag_at(h, unit), b = mag_at(l, unit);
    const int sa = h < 0.0, sb = l < 0.0;
    sadd128(a, a ? sa : 0, b, b ? sb : 0, m, sg);
    if (!m) sg = 0;
  };
  u128 xr, xi;
  int sr, si;
  comp(rh, rl, xr, sr);
  comp(ih, il, xi, si);
  return xint_norm(xr, sr, xi, si, unit + e + 126);
}

// a + b
__host__ __device__ __forceinline__ xint xint_add(const xint &a, const xint &b) {
  if (!a.x && !a.y) return b;
  if (!b.x && !b.y) return a;
  const xint &hi = a.e >= b.e ? a : b, &lo = a.e >= b.e ? b : a;
  const long long d = hi.e - lo.e;
  const u128 lx = d < 128 ? (lo.x >> d) : (u128)0, ly = d < 128 ? (lo.y >> d) : (u128)0;
  // operands below 2^127: halve both first so the sums cannot overflow
  u128 rx, ry;
  int sx, sy;
  sadd128(hi.x >> 1, hi.sx, lx >> 1, lo.sx, rx, sx);
  sadd128(hi.y >> 1, hi.sy, ly >> 1, lo.sy, ry, sy);
  return xint_norm(rx, rx ? sx : 0, ry, ry ? sy : 0, hi.e + 1);
}

// 1/m for a complex m with max(|mr|, |mi|) in [0.5, 1): an FP64 seed
// u0 = conj(m) / |m|^2 (relative error a few 2^-53), then one Newton step
// u = u0 + u0 (1 - m u0) in fixed point, which squares the seed's error:
// relative error about 2^-100.
__host__ __device__ __forceinline__ xint recip_xint(double mr, double mi) {
  const double inv = 1.0 / (mr * mr + mi * mi);
  const xint u0 = xint_from_dd2(mr * inv, 0.0, -mi * inv, 0.0, 0);
  const xint m = xint_from_dd2(mr, 0.0, mi, 0.0, 0);
  const xint one = xint_norm((u128)1 << 126, 0, 0, 0, 0);
  const xint e = xint_add(one, xint_neg(xint_mul(m, u0)));
  return xint_add(u0, xint_mul(u0, e));
}

// the output format (fpe_xc64: max(|re|, |im|) in [0.5, 1)) from a
// normalised xint, each component rounded to nearest at 53 bits
__host__ __device__ __forceinline__ fpe_xc64 xc64_from_xint(const xint &v) {
  fpe_xc64 o;
  if (!v.x && !v.y) {
    o.re = o.im = 0.0;
    o.e = 0;
    return o;
  }
  const unsigned long long hx = (unsigned long long)(v.x >> 74) + (unsigned long long)((v.x >> 73) & 1);
  const unsigned long long hy = (unsigned long long)(v.y >> 74) + (unsigned long long)((v.y >> 73) & 1);
  double re = (double)hx * 0x1p-53, im = (double)hy * 0x1p-53;  // exact: hx, hy <= 2^53
  o.e = v.e + 1;
  if (re == 1.0 || im == 1.0) {  // rounding carried into the next binade
    re *= 0.5;
    im *= 0.5;
    o.e += 1;
  }
  o.re = v.sx ? -re : re;
  o.im = v.sy ? -im : im;
  return o;
}

// z^n (n >= 0) as an xint with z's binary exponent folded in
__host__ __device__ __forceinline__ xint xint_pow_z(double zr, double zi, long long n, int f) {
  if (n <= 0) return xint_norm((u128)1 << 126, 0, 0, 0, 0);
#ifdef __CUDA_ARCH__
  xint r = xint_pow_unit(scale2(zr, -f), scale2(zi, -f), n);
#else
  xint r = xint_pow_unit(ldexp(zr, -f), ldexp(zi, -f), n);
#endif
  r.e += (long long)f * n;
  return r;
}

// the low 74 bits of a 128-bit magnitude, as a double scaled by 2^-74
__host__ __device__ __forceinline__ double low74_scaled(u128 x) {
  const unsigned long long lo = (unsigned long long)x, up = (unsigned long long)(x >> 64) & 0x3ffull;
  return (double)up * 0x1p-10 + (double)lo * 0x1p-74;
}

// extended double-double from a 128-bit mantissa pair
__host__ __device__ __forceinline__ xdd xdd_from_xint(const xint &v) {
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
  if (!v.x && !v.y) x.e = 0;
  return x;  // max(|rh|, |ih|) is in [0.5, 1) already: the larger top bit is at 126
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
// longer matters.  No FP64 instruction is used.
//
// The multiplier.  w = 2^beta z is used exactly, as w = i^q w' with w' in
// the closed first quadrant (a swap and sign changes of z's parts): each
// component of w' is its 53-bit mantissa as an unsigned 63-bit word.  When
// the two exponents are within 10 of each other (more for subnormals) both
// words share one exponent exactly; otherwise each keeps its own and the
// smaller component's products are shifted into the larger's frame (SPLIT).
// Horner with w = i^q w' runs as g_k = g_{k+1} w' + i^(-q m) b_k with
// m = top - k, and h = i^(q m) g at the end: rotating a coefficient by a
// power of i is a swap and sign changes, so no product carries a sign of w.
//
// The coefficients come packed (qpack): a 54-bit two's-complement mantissa
// and an exponent, placed into the frame with one variable shift.
//
// Magnitude budget: a product (x w) >> 64 with w < 2^63 has at most half
// the magnitude of x, so each component of h w' is at most max(|xr|, |xi|),
// and a coefficient adds less than 2^121 (larger ones move the frame up).
// From < 2^122 after normalising, eight steps stay below 2^125: callers
// normalise at least every eight steps.
// ---------------------------------------------------------------------------
typedef __int128 i128;

constexpr int kIsumTop = 121;        // top bit after normalising
constexpr int kIsumMaxSteps = 8;     // steps between normalisations
constexpr int kIsumCoefShift = 68;   // a coefficient 54-bit mantissa sits at most this far up

struct isum {
  i128 xr, xi;
  int G;
};

// frame of a zero sum: far below any coefficient, so the next nonzero
// coefficient sets the frame (and eight steps of a zero sum cannot wrap G)
constexpr int kIsumZeroFrame = -(1 << 29);

// w = i^q (w'r + i w'i), w'r = r 2^(E - dr), w'i = m 2^(E - di), r, m < 2^63
struct iw {
  uint32_t r0, r1, m0, m1;  // 32-bit limbs of the two words
  int dr, di, split, q;
  int E;
};

__host__ __device__ __forceinline__ int bitlen64(unsigned long long m) {
#ifdef __CUDA_ARCH__
  return m ? 64 - __clzll(m) : 0;
#else
  return m ? 64 - __builtin_clzll(m) : 0;
#endif
}

// |x| = m 2^e with m < 2^53 (m = 0 for x = 0)
__host__ __device__ __forceinline__ void decode_abs(double x, unsigned long long &m, int &e) {
  const unsigned long long bits = dbl_bits(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  m = bits & 0xfffffffffffffull;
  if (ex == 0) {
    e = -1074;
  } else {
    m |= 0x10000000000000ull;
    e = ex - 1075;
  }
}

__host__ __device__ __forceinline__ iw iw_from(double zr, double zi) {
  // z = i^q w' with Re w' > 0, Im w' >= 0 (z != 0)
  int q;
  double ar, ai;  // |parts| of w' in order (re, im)
  if (zr > 0.0 && zi >= 0.0) {
    q = 0, ar = zr, ai = zi;
  } else if (zr <= 0.0 && zi > 0.0) {
    q = 1, ar = zi, ai = -zr;
  } else if (zr < 0.0 && zi <= 0.0) {
    q = 2, ar = -zr, ai = -zi;
  } else {
    q = 3, ar = -zi, ai = zr;
  }
  unsigned long long mr, mi;
  int er, ei;
  decode_abs(ar, mr, er);
  decode_abs(ai, mi, ei);
  iw w;
  w.q = q;
  // each mantissa with its top bit at 62; exponents Er, Ei of the word's unit
  const int shr = mr ? 63 - bitlen64(mr) : 0, shi = mi ? 63 - bitlen64(mi) : 0;
  const int Er = er - shr, Ei = ei - shi;
  w.E = mr ? (mi ? (Er > Ei ? Er : Ei) : Er) : Ei;
  int dr = mr ? w.E - Er : 0, di = mi ? w.E - Ei : 0;
  // when the smaller word has that many trailing zeros it moves down exactly
  const int sdr = (dr > 0 && dr <= shr) ? dr : 0;
  const int sdi = (di > 0 && di <= shi) ? di : 0;
  const unsigned long long ur = (mr << shr) >> sdr, ui = (mi << shi) >> sdi;
  dr -= sdr;
  di -= sdi;
  w.r0 = (uint32_t)ur;
  w.r1 = (uint32_t)(ur >> 32);
  w.m0 = (uint32_t)ui;
  w.m1 = (uint32_t)(ui >> 32);
  w.dr = dr < 127 ? dr : 127;
  w.di = di < 127 ? di : 127;
  w.split = (w.dr | w.di) != 0;
  return w;
}

// x w / 2^64 for a two's-complement x (|x| < 2^127) and w = (w1:w0) < 2^63:
// the partial products of the two lowest 32-bit columns are dropped, so the
// result is within 3 of the exact quotient.  Computed on the unsigned bit
// pattern of x, then w 2^64 is subtracted when x < 0.
__host__ __device__ __forceinline__ i128 mulhi_limb(i128 xs, uint32_t w0, uint32_t w1) {
  const u128 x = (u128)xs;
  const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32), x2 = (uint32_t)(x >> 64), x3 = (uint32_t)(x >> 96);
  const uint32_t m = (uint32_t)((int32_t)x3 >> 31);
#ifdef __CUDA_ARCH__
  uint32_t r0, r1, r2, r3;
  asm("{\n\t"
      ".reg .u32 t0, t1;\n\t"
      "mul.hi.u32      %0, %5, %8;\n\t"        // col 2: hi(x1 w0)
      "mul.lo.u32      %1, %7, %8;\n\t"        // col 3: lo(x3 w0)
      "mul.hi.u32      %2, %7, %8;\n\t"        // col 4: hi(x3 w0)
      "mad.lo.cc.u32   %0, %6, %8, %0;\n\t"    // col 2 += lo(x2 w0)
      "madc.hi.cc.u32  %1, %6, %8, %1;\n\t"    // col 3 += hi(x2 w0)
      "addc.u32        %2, %2, 0;\n\t"
      "mad.lo.cc.u32   %0, %5, %9, %0;\n\t"    // col 2 += lo(x1 w1)
      "madc.lo.cc.u32  %1, %6, %9, %1;\n\t"    // col 3 += lo(x2 w1)
      "madc.lo.cc.u32  %2, %7, %9, %2;\n\t"    // col 4 += lo(x3 w1)
      "addc.u32        %3, 0, 0;\n\t"
      "mad.hi.cc.u32   %0, %4, %9, %0;\n\t"    // col 2 += hi(x0 w1)
      "madc.hi.cc.u32  %1, %5, %9, %1;\n\t"    // col 3 += hi(x1 w1)
      "madc.hi.cc.u32  %2, %6, %9, %2;\n\t"    // col 4 += hi(x2 w1)
      "madc.hi.u32     %3, %7, %9, %3;\n\t"    // col 5 += hi(x3 w1)
      "and.b32         t0, %8, %10;\n\t"       // x < 0: subtract w 2^64
      "and.b32         t1, %9, %10;\n\t"
      "sub.cc.u32      %2, %2, t0;\n\t"
      "subc.u32        %3, %3, t1;\n\t"
      "}"
      : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3)
      : "r"(x0), "r"(x1), "r"(x2), "r"(x3), "r"(w0), "r"(w1), "r"(m));
  return (i128)(((u128)r3 << 96) | ((u128)r2 << 64) | ((u128)r1 << 32) | (u128)r0);
#else
  // the same column sums, modulo 2^128
  auto lo = [](uint32_t a, uint32_t b) -> u128 { return (u128)(uint32_t)((uint64_t)a * b); };
  auto hi = [](uint32_t a, uint32_t b) -> u128 { return (u128)(uint32_t)(((uint64_t)a * b) >> 32); };
  u128 r = hi(x1, w0) + hi(x0, w1) + lo(x2, w0) + lo(x1, w1);
  r += (hi(x2, w0) + hi(x1, w1) + lo(x3, w0) + lo(x2, w1)) << 32;
  r += (hi(x3, w0) + hi(x2, w1) + lo(x3, w1)) << 64;
  r += hi(x3, w1) << 96;
  r -= ((u128)(((uint64_t)(w1 & m) << 32) | (w0 & m))) << 64;
  return (i128)r;
#endif
}

// a packed coefficient component: value = v 2^e
__host__ __device__ __forceinline__ void qdecode(unsigned long long q, long long &v, int &e) {
  v = (long long)(q << 10) >> 10;
  e = (int)(q >> 54) - kQBias;
}

// v 2^sh as a signed 128-bit value, sh <= kIsumCoefShift (truncated below 2^0)
__host__ __device__ __forceinline__ i128 place_q(long long v, int sh) {
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
  int er, ei;
  decode_abs(hr, mr, er);
  decode_abs(hm, mi, ei);
  isum h;
  if (!mr && !mi) {
    h.xr = h.xi = 0;
    h.G = kIsumZeroFrame;
    return h;
  }
  const int tr = mr ? er + bitlen64(mr) - 1 : -100000;
  const int ti = mi ? ei + bitlen64(mi) - 1 : -100000;
  h.G = (tr > ti ? tr : ti) - kIsumTop;
  const long long vr = hr < 0.0 ? -(long long)mr : (long long)mr;
  const long long vi = hm < 0.0 ? -(long long)mi : (long long)mi;
  h.xr = mr ? place_q(vr, er - h.G) : (i128)0;
  h.xi = mi ? place_q(vi, ei - h.G) : (i128)0;
  return h;
}

// multiply the fixed-point sum by i^t (exact)
__host__ __device__ __forceinline__ void isum_rotate(isum &h, int t) {
  const i128 r = h.xr, m = h.xi;
  switch (t & 3) {
    case 1: h.xr = -m, h.xi = r; break;
    case 2: h.xr = -r, h.xi = -m; break;
    case 3: h.xr = m, h.xi = -r; break;
    default: break;
  }
}

// g <- g w' 2^shift + i^t (br + i bi) from packed coefficient words, without
// normalising; CZ: complex w, CC: complex coefficient, SPLIT: w with two
// exponents.  we64 = w.E + shift + 64.  Returns nothing; t is the caller's.
template <bool CC, bool CZ, bool SPLIT>
__host__ __device__ __forceinline__ void isum_step(isum &h, const iw &w, int we64, unsigned long long qr,
                                                   unsigned long long qi, int t) {
  constexpr bool CH = CC || CZ;
  i128 re, im = 0;
  if (CZ) {
    i128 prr = mulhi_limb(h.xr, w.r0, w.r1), pir = mulhi_limb(h.xi, w.r0, w.r1);
    i128 pii = mulhi_limb(h.xi, w.m0, w.m1), pri = mulhi_limb(h.xr, w.m0, w.m1);
    if (SPLIT) {
      prr >>= w.dr, pir >>= w.dr;
      pii >>= w.di, pri >>= w.di;
    }
    re = prr - pii;
    im = pri + pir;
  } else {
    re = mulhi_limb(h.xr, w.r0, w.r1);
    if (CH) im = mulhi_limb(h.xi, w.r0, w.r1);
  }
  int G = h.G + we64;
  long long vr, vi = 0;
  int er, ei = -kQBias;
  qdecode(qr, vr, er);
  if (CC) qdecode(qi, vi, ei);
  if (CZ) {  // i^t (vr + i vi)
    if (t & 1) {
      const long long tv = vr;
      const int te = er;
      vr = vi, er = ei;
      vi = tv, ei = te;
    }
    if (t == 1 || t == 2) vr = -vr;
    if (t >= 2) vi = -vi;
  } else if (t & 2) {  // real w: t in {0, 2}
    vr = -vr;
    vi = -vi;
  }
  // a coefficient of 2^121 or more in this frame moves the frame up first
  const int etop = (er > ei ? er : ei) - kIsumCoefShift;
  const int need = etop > G ? etop : G;
  if (need > G) {
    const int d = need - G < 127 ? need - G : 127;
    re >>= d;
    im >>= d;
    G = need;
  }
  re += place_q(vr, er - G);
  if (CH) im += place_q(vi, ei - G);
  h.xr = re;
  h.xi = im;
  h.G = G;
}

// a fixed-point sum as a normalised xint (zero: the zero xint)
__host__ __device__ __forceinline__ xint xint_from_isum(const isum &h) {
  const int sr = h.xr < 0, si = h.xi < 0;
  const u128 ar = sr ? (u128)(-h.xr) : (u128)h.xr, ai = si ? (u128)(-h.xi) : (u128)h.xi;
  return xint_norm(ar, sr, ai, si, (long long)h.G + 126);
}

// extended double-double of a fixed-point sum
__device__ __forceinline__ xdd xdd_from_isum(const isum &h) { return xdd_from_xint(xint_from_isum(h)); }

// ---------------------------------------------------------------------------
// Extended values of the FP32 mode: an FP64 complex mantissa with an int64
// exponent, max(|r|, |i|) in [0.5, 1) or both zero.  Each operation rounds
// at a few 2^-53 relative, far below the mode's 2^-21 tolerance, and costs
// a third of the FP64 instructions of the double-double forms above.
// ---------------------------------------------------------------------------
struct xd {
  double r, i;
  long long e;
};

__device__ __forceinline__ xd xd_norm(double r, double i, long long e) {
  const double m = fmax(fabs(r), fabs(i));
  if (m == 0.0) return {0.0, 0.0, 0};
  const int f = frexp_exp(m);
  return {scale2(r, -f), scale2(i, -f), e + f};
}
__device__ __forceinline__ xd xd_mul(const xd &a, const xd &b) {
  return xd_norm(fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r), a.e + b.e);
}
// a * (zr + i zi) 2^ze
__device__ __forceinline__ xd xd_mul_d(const xd &a, double zr, double zi, long long ze) {
  return xd_norm(fma(a.r, zr, -a.i * zi), fma(a.r, zi, a.i * zr), a.e + ze);
}
__device__ __forceinline__ xd xd_add(const xd &a, const xd &b) {
  if (a.r == 0.0 && a.i == 0.0) return b;
  if (b.r == 0.0 && b.i == 0.0) return a;
  if (a.e >= b.e) {
    const int d = (int)max(-2000LL, b.e - a.e);
    return xd_norm(a.r + scale2(b.r, d), a.i + scale2(b.i, d), a.e);
  }
  const int d = (int)max(-2000LL, a.e - b.e);
  return xd_norm(b.r + scale2(a.r, d), b.i + scale2(a.i, d), b.e);
}
__device__ __forceinline__ xdd xdd_from_xd(const xd &x) { return {x.r, 0.0, x.i, 0.0, x.e}; }

// z^n (n >= 0) on the integer pipe, kept to its top 53 bits
__device__ __forceinline__ xd xd_pow_int(double zr, double zi, long long n) {
  if (n <= 0) return {0.5, 0.0, 1};
  const int f = frexp_exp(fmax(fabs(zr), fabs(zi)));
  const xint v = xint_pow_unit(scale2(zr, -f), scale2(zi, -f), n);
  // component = X 2^(e - 126) with X < 2^127: its top bits H = X >> 74 times 2^(e - 52)
  const double hr = (double)(unsigned long long)(v.x >> 74), hi = (double)(unsigned long long)(v.y >> 74);
  return xd_norm(v.sx ? -hr : hr, v.sy ? -hi : hi, v.e - 52 + (long long)f * n);
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

// ---------------------------------------------------------------------------
// Lists a long-window point and reserves its warp groups: group 0 lives in
// slot i (its list index), groups 1.. in extra slots; when the extra slots run
// out the window gets one group and the slots of its failed reservation that
// exist are marked unused (-1).
__device__ __forceinline__ void list_long_window(long long L, long long span, uint32_t pos, uint32_t *cnt,
                                                 int32_t *long_list, int32_t *long_ngroups, int32_t *long_gbase,
                                                 int32_t *extra_owner, int32_t *extra_group, int extra_cap) {
  uint32_t i = atomicAdd(&cnt[kCntLong], 1u);
  long_list[i] = (int32_t)pos;
  int ng = (int)min((L + span - 1) / span, 0x7fffLL);  // the upper 16 bits count finished groups
  int gb = 0;
  if (ng > 1) {
    gb = (int)atomicAdd(&cnt[kCntExtra], (uint32_t)(ng - 1));
    if (gb + ng - 1 > extra_cap) {
      for (int g = 1; g < ng && gb + g - 1 < extra_cap; ++g) extra_owner[gb + g - 1] = -1;
      ng = 1;
    } else {
      for (int g = 1; g < ng; ++g) {
        extra_owner[gb + g - 1] = (int32_t)i;
        extra_group[gb + g - 1] = g;
      }
    }
  }
  long_ngroups[i] = ng;
  long_gbase[i] = gb;
}

}  // namespace fpe
