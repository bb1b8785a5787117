// Host build of the integer-pipe Horner step (fpe_device.cuh) for a CPU test
// against exact rational arithmetic.  Compiled by tests/test_int_horner_host.py.
#include "fpe_device.cuh"
using namespace fpe;

template <bool CC, bool CZ, bool SPLIT>
static void run(isum &h, const iw &w, const double *br, const double *bi, int n) {
  const int dq = (4 - w.q) & 3;
  int t = dq, c = 0;
  for (int k = n - 2; k >= 0; --k) {
    isum_step<CC, CZ, SPLIT>(h, w, w.E + 64, qpack(br[k]), CC ? qpack(bi[k]) : 0ull, t);
    t = (t + dq) & 3;
    if (++c == kIsumMaxSteps) {
      isum_normalise(h);
      c = 0;
    }
  }
  isum_normalise(h);
  isum_rotate(h, (w.q * ((n - 1) & 3)) & 3);
}

// top-down Horner h = b[n-1]; h = h z + b[k] as the kernels run it;
// returns |xr|, |xi| as 64-bit limbs, the signs, G, and whether w was split
extern "C" int int_horner(const double *br, const double *bi, int n, double zr, double zi, int complex_z,
                          int complex_c, unsigned long long *out, int *signs, long long *G) {
  isum h = isum_from(br[n - 1], complex_c ? bi[n - 1] : 0.0);
  const iw w = iw_from(zr, complex_z ? zi : 0.0);
  if (complex_z && complex_c) {
    if (w.split) run<true, true, true>(h, w, br, bi, n);
    else run<true, true, false>(h, w, br, bi, n);
  } else if (complex_z) {
    if (w.split) run<false, true, true>(h, w, br, bi, n);
    else run<false, true, false>(h, w, br, bi, n);
  } else if (complex_c) {
    run<true, false, false>(h, w, br, bi, n);
  } else {
    run<false, false, false>(h, w, br, bi, n);
  }
  const u128 ar = h.xr < 0 ? (u128)(-h.xr) : (u128)h.xr, ai = h.xi < 0 ? (u128)(-h.xi) : (u128)h.xi;
  out[0] = (unsigned long long)ar;
  out[1] = (unsigned long long)(ar >> 64);
  out[2] = (unsigned long long)ai;
  out[3] = (unsigned long long)(ai >> 64);
  signs[0] = h.xr < 0;
  signs[1] = h.xi < 0;
  *G = h.G;
  return w.split;
}
