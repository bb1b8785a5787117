/*
 * CPU ORACLE -- test infrastructure only.  Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path.
 *
 * Plain, slow, obviously correct polynomial evaluation in extended
 * double-double arithmetic: a value is ((re_hi + re_lo) + i (im_hi + im_lo)) * 2^e
 * with e a 64-bit integer, so neither huge coefficients (beyond the FP64
 * range) nor huge |z|^d overflow, and the mantissa carries about 106 bits.
 *
 * The error-free transformations are the published ones: TwoSum (Knuth,
 * TAOCP vol. 2, 4.2.2) and the FMA-based TwoProd.  The paper measures FPE's
 * accuracy against a much higher-precision Horner evaluation (§8.3, accuracy
 * benchmark); oracle_horner is that reference at ~106 bits.
 *
 * Functions:
 *   oracle_horner      P(z) = sum_{k=0}^{d} a_k z^k by Horner's scheme over every
 *                      term (Horner's scheme, §1), plus S(z) = sum |a_k||z|^k and
 *                      log2 max_k |a_k z^k| (the M of Thm. equivAlgo).
 *   oracle_window_sum  Q(z) = sum over k in [lo, hi] with good[k] of a_k z^k
 *                      (eq. reducedQlambda), evaluated as z^lo times a Horner sum
 *                      over the window, z^lo by repeated squaring (§8.2).
 *   oracle_window_sum_fp64
 *                      the same sum with the Horner steps in plain FP64 complex
 *                      arithmetic and a 64-bit binary exponent (renormalised when
 *                      the partial sum leaves [2^-400, 2^400]), z^lo by repeated
 *                      squaring in double-double: Algorithm A_p's evaluation as a
 *                      plain CPU program in hardware floats (the paper's p = 53
 *                      runs, §8.3), timed as a CPU baseline.
 *   oracle_set_threads the number of OpenMP threads of the calls above.
 *
 * Coefficients: a_k = ((are[k] + are_lo[k]) + i (aim[k] + aim_lo[k])) * 2^ae[k];
 * aim, are_lo, aim_lo, ae may be NULL (zero).  Points: zim may be NULL (real).
 * Output per point j: out[4j..4j+3] = re_hi, re_lo, im_hi, im_lo; oute[j] = e.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; int64_t e; } xdd; /* (re + i im) * 2^e */

static dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb);
  dd r = {s, err};
  return r;
}
static dd quick_two_sum(double a, double b) { /* requires |a| >= |b| or a == 0 */
  double s = a + b;
  dd r = {s, b - (s - a)};
  return r;
}
static dd two_prod(double a, double b) {
  double p = a * b;
  dd r = {p, fma(a, b, -p)};
  return r;
}
static dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static dd dd_ldexp(dd a, int k) { dd r = {ldexp(a.hi, k), ldexp(a.lo, k)}; return r; }
static int dd_is_zero(dd a) { return a.hi == 0.0 && a.lo == 0.0; }

/* renormalise so that max(|re.hi|, |im.hi|) lies in [0.5, 1), or all zero */
static xdd xdd_norm(xdd x) {
  double m = fmax(fabs(x.re.hi), fabs(x.im.hi));
  if (m == 0.0) {
    if (!dd_is_zero(x.re) || !dd_is_zero(x.im)) { /* hi zero but lo not: fold */
      x.re = quick_two_sum(x.re.lo, 0.0);
      x.im = quick_two_sum(x.im.lo, 0.0);
      m = fmax(fabs(x.re.hi), fabs(x.im.hi));
      if (m == 0.0) { x.e = 0; return x; }
    } else {
      x.e = 0;
      return x;
    }
  }
  int f;
  frexp(m, &f);
  x.re = dd_ldexp(x.re, -f);
  x.im = dd_ldexp(x.im, -f);
  x.e += f;
  return x;
}
static int xdd_is_zero(xdd x) { return dd_is_zero(x.re) && dd_is_zero(x.im); }

/* x + y for extended values */
static xdd xdd_add(xdd x, xdd y) {
  if (xdd_is_zero(x)) return xdd_norm(y);
  if (xdd_is_zero(y)) return xdd_norm(x);
  x = xdd_norm(x);
  y = xdd_norm(y);
  if (x.e < y.e) { xdd t = x; x = y; y = t; }
  int64_t sh = y.e - x.e; /* <= 0 */
  if (sh < -2200) return x; /* y below 2^-2100 of x: beyond any precision here */
  y.re = dd_ldexp(y.re, (int)sh);
  y.im = dd_ldexp(y.im, (int)sh);
  xdd r = {dd_add(x.re, y.re), dd_add(x.im, y.im), x.e};
  return xdd_norm(r);
}
/* x * y for extended values */
static xdd xdd_mul(xdd x, xdd y) {
  xdd r;
  r.re = dd_add(dd_mul(x.re, y.re), dd_neg(dd_mul(x.im, y.im)));
  r.im = dd_add(dd_mul(x.re, y.im), dd_mul(x.im, y.re));
  r.e = x.e + y.e;
  return xdd_norm(r);
}
static xdd xdd_from(double re, double re_lo, double im, double im_lo, int64_t e) {
  xdd r;
  r.re = two_sum(re, re_lo);
  r.im = two_sum(im, im_lo);
  r.e = e;
  return xdd_norm(r);
}
/* z^n by repeated squaring (n >= 0) */
static xdd xdd_pow(xdd z, int64_t n) {
  xdd r = xdd_from(1.0, 0.0, 0.0, 0.0, 0);
  xdd b = z;
  while (n > 0) {
    if (n & 1) r = xdd_mul(r, b);
    n >>= 1;
    if (n) b = xdd_mul(b, b);
  }
  return r;
}

static xdd coef(int64_t k, const double *are, const double *aim, const double *are_lo,
                const double *aim_lo, const int64_t *ae) {
  return xdd_from(are[k], are_lo ? are_lo[k] : 0.0, aim ? aim[k] : 0.0, aim_lo ? aim_lo[k] : 0.0,
                  ae ? ae[k] : 0);
}

/* Horner from index hi down to lo: returns sum_{k=lo}^{hi} [mask] a_k z^{k-lo} */
static xdd horner_range(int64_t lo, int64_t hi, xdd z, const double *are, const double *aim,
                        const double *are_lo, const double *aim_lo, const int64_t *ae,
                        const uint8_t *good) {
  xdd h = xdd_from(0.0, 0.0, 0.0, 0.0, 0);
  for (int64_t k = hi; k >= lo; --k) {
    if (!xdd_is_zero(h)) h = xdd_mul(h, z);
    if (good && !good[k]) continue;
    h = xdd_add(h, coef(k, are, aim, are_lo, aim_lo, ae));
  }
  return h;
}

static void store(xdd v, int64_t j, double *out, int64_t *oute) {
  v = xdd_norm(v);
  out[4 * j + 0] = v.re.hi;
  out[4 * j + 1] = v.re.lo;
  out[4 * j + 2] = v.im.hi;
  out[4 * j + 3] = v.im.lo;
  oute[j] = v.e;
}

void oracle_horner(int64_t n_coef, const double *are, const double *aim, const double *are_lo,
                   const double *aim_lo, const int64_t *ae, int64_t npts, const double *zre,
                   const double *zim, double *out, int64_t *oute, double *S_m, int64_t *S_e,
                   double *log2M) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < npts; ++j) {
    xdd z = xdd_from(zre[j], 0.0, zim ? zim[j] : 0.0, 0.0, 0);
    xdd h = horner_range(0, n_coef - 1, z, are, aim, are_lo, aim_lo, ae, NULL);
    store(h, j, out, oute);
    /* S(z) = sum |a_k| |z|^k in extended FP64 (a tolerance scale: a few ulps suffice) */
    double az = hypot(zre[j], zim ? zim[j] : 0.0);
    int fz;
    double mz = frexp(az, &fz);
    double sm = 0.0;
    int64_t se = 0;
    double best = -INFINITY;
    double lz = (az > 0.0) ? log2(az) : -INFINITY;
    for (int64_t k = n_coef - 1; k >= 0; --k) {
      /* s <- s * |z| */
      if (sm != 0.0) {
        sm *= mz;
        se += fz;
      }
      double ar = are[k] + (are_lo ? are_lo[k] : 0.0);
      double ai = (aim ? aim[k] : 0.0) + (aim_lo ? aim_lo[k] : 0.0);
      double am = hypot(ar, ai);
      if (am != 0.0) {
        int64_t e = ae ? ae[k] : 0;
        double t = lz == -INFINITY ? (k == 0 ? log2(am) + (double)e : -INFINITY)
                                   : log2(am) + (double)e + (double)k * lz;
        if (t > best) best = t;
        int fa;
        double ma = frexp(am, &fa);
        int64_t ea = e + fa;
        if (sm == 0.0) {
          sm = ma;
          se = ea;
        } else {
          int64_t sh = ea - se;
          if (sh > 1000) {
            sm = ma;
            se = ea;
          } else if (sh >= -1100) {
            sm += ldexp(ma, (int)sh);
          }
        }
      }
      if (sm != 0.0) {
        int f;
        sm = frexp(sm, &f);
        se += f;
      }
    }
    S_m[j] = sm;
    S_e[j] = se;
    log2M[j] = best;
  }
}

/* S over a window: sum over k in [lo, hi] with good[k] of |a_k| |z|^k, as (m, e) */
static void window_abs_sum(int64_t lo, int64_t hi, double az, const double *are, const double *aim,
                           const double *are_lo, const double *aim_lo, const int64_t *ae,
                           const uint8_t *good, double *Sm, int64_t *Se) {
  double sm = 0.0;
  int64_t se = 0;
  int fz;
  double mz = frexp(az, &fz);
  for (int64_t k = hi; k >= lo; --k) {
    if (sm != 0.0) { /* s <- s |z|, renormalised at once: a run of skipped terms must not
                        let the mantissa drift toward the subnormal range */
      int f;
      sm = frexp(sm * mz, &f);
      se += fz + f;
    }
    if (good && !good[k]) continue;
    double ar = are[k] + (are_lo ? are_lo[k] : 0.0);
    double ai = (aim ? aim[k] : 0.0) + (aim_lo ? aim_lo[k] : 0.0);
    double am = hypot(ar, ai);
    if (am == 0.0) continue;
    int fa;
    double ma = frexp(am, &fa);
    int64_t ea = (ae ? ae[k] : 0) + fa;
    if (sm == 0.0) {
      sm = ma;
      se = ea;
    } else {
      int64_t sh = ea - se;
      if (sh > 1000) { /* the sum so far is below 2^-999 of this term */
        sm = ma;
        se = ea;
      } else if (sh >= -1100) {
        sm += ldexp(ma, (int)sh);
      }
    }
    int f;
    sm = frexp(sm, &f);
    se += f;
  }
  if (sm != 0.0 && lo > 0) { /* times |z|^lo = 2^(lo log2|z|) */
    double t = (double)lo * log2(az);
    double fl = floor(t);
    sm *= exp2(t - fl);
    int f;
    sm = frexp(sm, &f);
    se += (int64_t)fl + f;
  }
  *Sm = sm;
  *Se = se;
}

void oracle_window_sum(int64_t n_coef, const double *are, const double *aim, const double *are_lo,
                       const double *aim_lo, const int64_t *ae, const uint8_t *good, int64_t npts,
                       const double *zre, const double *zim, const int64_t *lo, const int64_t *hi,
                       double *out, int64_t *oute, double *S_m, int64_t *S_e) {
  (void)n_coef;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < npts; ++j) {
    xdd z = xdd_from(zre[j], 0.0, zim ? zim[j] : 0.0, 0.0, 0);
    xdd v;
    double sm = 0.0;
    int64_t se = 0;
    if (hi[j] < lo[j]) {
      v = xdd_from(0.0, 0.0, 0.0, 0.0, 0);
    } else {
      xdd h = horner_range(lo[j], hi[j], z, are, aim, are_lo, aim_lo, ae, good);
      v = xdd_mul(h, xdd_pow(z, lo[j]));
      if (S_m) window_abs_sum(lo[j], hi[j], hypot(zre[j], zim ? zim[j] : 0.0), are, aim, are_lo, aim_lo, ae,
                              good, &sm, &se);
    }
    store(v, j, out, oute);
    if (S_m) {
      S_m[j] = sm;
      S_e[j] = se;
    }
  }
}

/* the FP64 restatement: sum_{k in [lo, hi], good[k]} a_k z^k */
void oracle_window_sum_fp64(int64_t n_coef, const double *are, const double *aim, const int64_t *ae,
                            const uint8_t *good, int64_t npts, const double *zre, const double *zim,
                            const int64_t *lo, const int64_t *hi, double *out, int64_t *oute) {
  (void)n_coef;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < npts; ++j) {
    const double zr = zre[j], zi = zim ? zim[j] : 0.0;
    double hr = 0.0, hm = 0.0;
    int64_t E = 0; /* value = (hr + i hm) 2^E */
    for (int64_t k = hi[j]; k >= lo[j] && hi[j] >= lo[j]; --k) {
      const double nr = hr * zr - hm * zi, ni = hr * zi + hm * zr; /* h <- h z */
      hr = nr;
      hm = ni;
      if (good && !good[k]) continue;
      double br = are[k], bi = aim ? aim[k] : 0.0;
      if (br == 0.0 && bi == 0.0) continue;
      const int64_t e = ae ? ae[k] : 0;
      if (hr == 0.0 && hm == 0.0) {
        E = e; /* the first term sets the frame */
      } else if (e - E > 300) { /* a term far above the frame moves the frame up to it */
        const int64_t sh = E - e < -2000 ? -2000 : E - e;
        hr = ldexp(hr, (int)sh);
        hm = ldexp(hm, (int)sh);
        E = e;
      }
      const int64_t d = e - E; /* <= 300: the coefficient in the frame 2^E */
      if (d != 0) {
        const int64_t dd_ = d < -2000 ? -2000 : d;
        br = ldexp(br, (int)dd_);
        bi = ldexp(bi, (int)dd_);
      }
      hr += br;
      hm += bi;
      const double m = fmax(fabs(hr), fabs(hm));
      if (m != 0.0 && (m > 0x1p400 || m < 0x1p-400)) {
        int f;
        frexp(m, &f);
        hr = ldexp(hr, -f);
        hm = ldexp(hm, -f);
        E += f;
      }
    }
    xdd h = xdd_from(hr, 0.0, hm, 0.0, E);
    xdd v = xdd_is_zero(h) ? h : xdd_mul(h, xdd_pow(xdd_from(zr, 0.0, zi, 0.0, 0), lo[j]));
    store(v, j, out, oute);
  }
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
