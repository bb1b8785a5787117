// Host build of the fixed-point bookkeeping helpers (fpe_device.cuh) for a
// CPU test against exact rational arithmetic.  Compiled by tests/test_xint_host.py.
#include "fpe_device.cuh"
using namespace fpe;

static void put(const xint &v, unsigned long long *o, int *s, long long *e) {
  o[0] = (unsigned long long)v.x;
  o[1] = (unsigned long long)(v.x >> 64);
  o[2] = (unsigned long long)v.y;
  o[3] = (unsigned long long)(v.y >> 64);
  s[0] = v.sx;
  s[1] = v.sy;
  *e = v.e;
}

// value = ((-1)^s0 X + i (-1)^s1 Y) 2^(e - 126)
extern "C" void t_recip(double mr, double mi, unsigned long long *o, int *s, long long *e) {
  put(recip_xint(mr, mi), o, s, e);
}
extern "C" void t_from_dd2(double rh, double rl, double ih, double il, long long e0, unsigned long long *o, int *s,
                           long long *e) {
  put(xint_from_dd2(rh, rl, ih, il, e0), o, s, e);
}
extern "C" void t_add(double ar, double ai, long long ae, double br, double bi, long long be, unsigned long long *o,
                      int *s, long long *e) {
  put(xint_add(xint_from_dd2(ar, 0.0, ai, 0.0, ae), xint_from_dd2(br, 0.0, bi, 0.0, be)), o, s, e);
}
extern "C" void t_pow_out(double zr, double zi, long long n, double *re, double *im, long long *e) {
  int f = 0;
  frexp(fabs(zr) > fabs(zi) ? zr : zi, &f);
  const fpe_xc64 v = xc64_from_xint(xint_pow_z(zr, zi, n, f));
  *re = v.re;
  *im = v.im;
  *e = v.e;
}
