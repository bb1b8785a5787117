// Device arithmetic for the FPE kernels: power-of-two scaling by exponent-field
// construction, double-double error-free transformations (TwoSum: Knuth,
// TAOCP 4.2.2; TwoProd via FMA), and an extended-exponent complex
// double-double type used for the valuation monomial z^l (§8.2) and for
// combining partial window sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
