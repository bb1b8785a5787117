// Host build of the tensor-core path's integer arithmetic (fpe_tc_arith.cuh)
// for a CPU test against exact integers and rationals.  Compiled by
// tests/test_tc_arith_host.py.
#include "fpe_tc_arith.cuh"
using namespace fpe;

static u128 mk(const unsigned long long *w) { return ((u128)w[1] << 64) | w[0]; }

// the ten bf16 digits of F (< 2^69) with sign neg, and the same pair word's high half
extern "C" void t_digits(const unsigned long long *f, unsigned neg, unsigned short *lo, unsigned short *hi) {
  uint32_t x[kSl];
  bchunks70(mk(f), x);
  const DigitSign s = digit_sign(neg);
  for (int j = 0; j < kSl; ++j) {
    const uint32_t w = bf16_pair(x[j], s, x[j], s);
    lo[j] = (unsigned short)(w & 0xffffu);
    hi[j] = (unsigned short)(w >> 16);
  }
}

// sum_t v_t 128^(9 - t) from ten fp32 accumulators (exact integers)
extern "C" void t_join(const float *v, unsigned long long *mag, int *neg) {
  float acc[kAcc];
  for (int t = 0; t < kAcc; ++t) acc[t] = v[t];
  u128 m;
  join_vals(acc, m, *neg);
  mag[0] = (unsigned long long)m;
  mag[1] = (unsigned long long)(m >> 64);
}

// One output row of one block as the MMAs compute it: a 64-long dot product
// of A' row digits with Z' column digits, the digit pairs (s, s') with
// s + s' = t <= 9 added into accumulator t in fp32 (the order below; the
// tensor core's differs, which is harmless while every partial sum is an
// exact integer), then joined.  a[k], z[k] (k < 64) are 69-bit magnitudes
// (two words each) with signs; exact[t] receives the same sums in 64-bit
// integers, so the caller can check that fp32 lost nothing.
extern "C" void t_row(const unsigned long long *a, const int *as, const unsigned long long *z, const int *zs,
                      unsigned long long *mag, int *neg, long long *exact) {
  float acc[kAcc];
  long long ex[kAcc];
  for (int t = 0; t < kAcc; ++t) {
    acc[t] = 0.0f;
    ex[t] = 0;
  }
  for (int k = 0; k < 2 * kTB; ++k) {
    uint32_t xa[kSl], xz[kSl];
    bchunks70(mk(a + 2 * k), xa);
    bchunks70(mk(z + 2 * k), xz);
    const DigitSign sa = digit_sign((uint32_t)as[k]), sz = digit_sign((uint32_t)zs[k]);
    float da[kSl], dz[kSl];
    for (int j = 0; j < kSl; ++j) {
      da[j] = fmaf(tc_bitsf(xa[j]), sa.s, sa.k);
      dz[j] = fmaf(tc_bitsf(xz[j]), sz.s, sz.k);
    }
    for (int s = 0; s < kSl; ++s)
      for (int s2 = 0; s2 < kSl - s; ++s2) {
        acc[s + s2] += da[s] * dz[s2];  // a product of two digits is exact in fp32
        ex[s + s2] += (long long)da[s] * (long long)dz[s2];
      }
  }
  for (int t = 0; t < kSl; ++t) exact[t] = ex[t];
  u128 m;
  join_vals(acc, m, *neg);
  mag[0] = (unsigned long long)m;
  mag[1] = (unsigned long long)(m >> 64);
  for (int t = 0; t < kSl; ++t) exact[kSl + t] = (long long)acc[t];
}

static void put_xh(const xh &v, unsigned long long *m, int *s, long long *e) {
  m[0] = v.x;
  m[1] = v.y;
  s[0] = v.sx;
  s[1] = v.sy;
  *e = v.e;
}

static xh get_xh(const unsigned long long *m, const int *s, long long e) {
  return xh_norm(m[0], s[0], m[1], s[1], e);
}

// value = ((-1)^s0 m0 + i (-1)^s1 m1) 2^(e - 63)
extern "C" void t_xh_mul(const unsigned long long *am, const int *as, long long ae, const unsigned long long *bm,
                         const int *bs, long long be, unsigned long long *m, int *s, long long *e) {
  put_xh(xh_mul(get_xh(am, as, ae), get_xh(bm, bs, be)), m, s, e);
}
extern "C" void t_xh_add(const unsigned long long *am, const int *as, long long ae, const unsigned long long *bm,
                         const int *bs, long long be, unsigned long long *m, int *s, long long *e) {
  put_xh(xh_add(get_xh(am, as, ae), get_xh(bm, bs, be)), m, s, e);
}
// from a 128-bit magnitude pair (value X 2^(e - 126))
extern "C" void t_xh_from128(const unsigned long long *x, int sx, const unsigned long long *y, int sy, long long e,
                             unsigned long long *m, int *s, long long *eo) {
  put_xh(xh_from128(mk(x), sx, mk(y), sy, e), m, s, eo);
}
