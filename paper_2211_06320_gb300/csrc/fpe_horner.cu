// The plain form beside FPE: Horner's scheme over all d+1 coefficients (§1),
// one thread per point, on the same rescaled coefficients b_k = a_k 2^-rho(k)
// (pieces of constant integer slope, w_j = 2^beta_j z) as the FPE kernels.
// Outside a point's window the partial sums can outgrow the FP64 range, so
// the running value carries an extra exponent E (value = h 2^(rho(k) + E)):
// every few terms h is renormalised when it passes 2^512, and while E > 0 each
// coefficient enters scaled by 2^-E.
//
// compensated = true runs compensated Horner: each step's rounding errors are
// captured exactly by error-free transformations (TwoProd via FMA, TwoSum)
// and accumulated by a second Horner recurrence c <- c w + errors, and the
// result is h + c (the compensated Horner schemes cited in §1).
#include <cuda_runtime.h>

#include "fpe_device.cuh"
#include "fpe_internal.h"

namespace fpe {

template <bool CC, bool CZ, bool COMP>
__global__ void __launch_bounds__(128) k_horner(DevPoly P, int n, const double *__restrict__ zre,
                                                const double *__restrict__ zim, fpe_xc64 *__restrict__ out,
                                                int32_t *status) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double zr = zre[p], zi = CZ ? zim[p] : 0.0;
  fpe_xc64 o;
  if (!isfinite(zr) || !isfinite(zi)) {
    o.re = o.im = __longlong_as_double(0x7ff8000000000000ll);
    o.e = 0;
    atomicOr(status, kStatusNonFinite);
    out[p] = o;
    return;
  }
  if (zr == 0.0 && zi == 0.0) {
    o.re = P.a0_re;
    o.im = P.a0_im;
    o.e = (P.a0_re == 0.0 && P.a0_im == 0.0) ? 0 : P.a0_e;
    out[p] = o;
    return;
  }
  const double *__restrict__ b = P.b_full;
  const long long D = P.D;
  int j = P.npieces - 1;
  double hr, hm;
  if (CC) {
    double2 c = reinterpret_cast<const double2 *>(b)[D];
    hr = c.x;
    hm = c.y;
  } else {
    hr = b[D];
    hm = 0.0;
  }
  double cr = 0.0, cm = 0.0;  // compensation (COMP only)
  long long E = 0;
  long long k = D - 1;
  while (k >= 0) {
    const int k0 = P.piece_k0[j];
    const int beta = P.piece_beta[j];
    const double wr = scale2(zr, beta), wi = CZ ? scale2(zi, beta) : 0.0;
    // terms between renormalisation checks: |w|^R stays below 2^400
    const int lw = frexp_exp(fmax(fabs(wr), fabs(wi)) + 1e-300);
    const int R = max(1, min(32, 400 / max(1, abs(lw) + 1)));
    while (k >= k0) {
      const long long kstop = max((long long)k0, k - R + 1);
      const double sc = E == 0 ? 1.0 : (E > 1100 ? 0.0 : scale2(1.0, -(int)E));
      for (; k >= kstop; --k) {
        double br, bi;
        if (CC) {
          double2 c = __ldg(reinterpret_cast<const double2 *>(b) + k);
          br = c.x * sc;
          bi = c.y * sc;
        } else {
          br = __ldg(b + k) * sc;
          bi = 0.0;
        }
        horner_step<CC, CZ, COMP>(hr, hm, cr, cm, wr, wi, br, bi);
      }
      // renormalise when |h| passes 2^512
      double m = fmax(fabs(hr), fabs(hm));
      if (m > 0x1p512) {
        int f = frexp_exp(m);
        double s = scale2(1.0, -f);
        hr *= s;
        hm *= s;
        cr *= s;
        cm *= s;
        E += f;
      }
    }
    if (k < 0) break;
    --j;  // entering piece j from j + 1
    const double s = pow2i(P.piece_delta[j]);
    hr *= s;
    hm *= s;
    cr *= s;
    cm *= s;
  }
  // value = (h + c) 2^(rho(0) + E) z^v
  const long long rho0 = P.piece_rho0[0];
  xdd v;
  {
    dd r = two_sum(hr, cr), i = two_sum(hm, cm);
    xdd x = {r.hi, r.lo, i.hi, i.lo, rho0 + E};
    v = xdd_norm(x);
  }
  if (P.v > 0) v = xdd_mul(v, xdd_pow_int(zr, zi, P.v));
  out[p] = xdd_out(v);
}

fpe_status launch_horner(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n64, fpe_xc64 *out,
                         int compensated, cudaStream_t st) {
  if (n64 == 0) return FPE_OK;
  const int n = (int)n64;
  const bool cz = z_im != nullptr, cc = P->complex_coef;
  const int nb = (n + 127) / 128;
  ProfScope ps(compensated ? "k_horner_comp" : "k_horner_plain", st);
#define FPE_HORNER_LAUNCH(CCv, CZv, COMPv) \
  k_horner<CCv, CZv, COMPv><<<nb, 128, 0, st>>>(P->dev, n, z_re, z_im, out, P->d_status)
  if (compensated) {
    if (cc && cz) FPE_HORNER_LAUNCH(true, true, true);
    else if (cc) FPE_HORNER_LAUNCH(true, false, true);
    else if (cz) FPE_HORNER_LAUNCH(false, true, true);
    else FPE_HORNER_LAUNCH(false, false, true);
  } else {
    if (cc && cz) FPE_HORNER_LAUNCH(true, true, false);
    else if (cc) FPE_HORNER_LAUNCH(true, false, false);
    else if (cz) FPE_HORNER_LAUNCH(false, true, false);
    else FPE_HORNER_LAUNCH(false, false, false);
  }
#undef FPE_HORNER_LAUNCH
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_horner launch");
  return FPE_OK;
}

}  // namespace fpe
