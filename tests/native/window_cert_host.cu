// Host build of the certified FP64 window sums (fpe_window.cuh) for a CPU
// test against exact rational sums.  Compiled by tests/test_window_cert_host.py.
#include <vector>

#include "fpe_window.cuh"
using namespace fpe;

static std::vector<float> g_bmag;

// the handle's view of the coefficients b (n of them); bmag as preconditioning makes it
static DevPoly make_poly(const double *b, int cc, const int32_t *k0, const int32_t *beta, const int32_t *delta,
                         const int64_t *rho0, const int32_t *first, int npieces, int log2_piece) {
  DevPoly P;
  memset(&P, 0, sizeof P);
  const int n = k0[npieces];
  g_bmag.resize(n);
  for (int k = 0; k < n; ++k) g_bmag[k] = coef_mag_lo(cc ? b[2 * k] : b[k], cc ? b[2 * k + 1] : 0.0);
  P.bmag = g_bmag.data();
  P.b = b;
  P.piece_k0 = k0;
  P.piece_beta = beta;
  P.piece_delta = delta;
  P.piece_rho0 = rho0;
  P.piece_first = first;
  P.npieces = npieces;
  P.log2_piece = log2_piece;
  P.complex_coef = cc;
  return P;
}

// top-down pass over [lo, hi]: out = (hr, hm), *rho = rho(lo), es = (E, S); returns ok
extern "C" int wc_top(const double *b, int cc, int cz, const int32_t *k0, const int32_t *beta, const int32_t *delta,
                      const int64_t *rho0, const int32_t *first, int npieces, int log2_piece, double zr, double zi,
                      long long lo, long long hi, double *out, long long *rho, float *es) {
  const DevPoly P = make_poly(b, cc, k0, beta, delta, rho0, first, npieces, log2_piece);
  Cert ct;
  if (!cz) zi = 0.0;
  if (cc && cz) window_horner<true, true>(P, P.b, zr, zi, lo, hi, out[0], out[1], *rho, ct);
  else if (cc) window_horner<true, false>(P, P.b, zr, zi, lo, hi, out[0], out[1], *rho, ct);
  else if (cz) window_horner<false, true>(P, P.b, zr, zi, lo, hi, out[0], out[1], *rho, ct);
  else window_horner<false, false>(P, P.b, zr, zi, lo, hi, out[0], out[1], *rho, ct);
  es[0] = ct.E;
  es[1] = ct.S;
  return ct.ok;
}

template <bool CC, bool CZ>
static void rev(const DevPoly &P, double zr, double zi, long long lo, long long hi, int blocks, double *out,
                long long *rho, Cert &ct) {
  // the reciprocal and its powers as the evaluation kernels form them
  int f;
  frexp(fmax(fabs(zr), fabs(zi)), &f);
  const double mr = ldexp(zr, -f), mi = ldexp(zi, -f);
  const xint u = recip_xint(mr, mi);
  const xdd u1 = xdd_from_xint(u);
  const xint u2 = xint_sqr(u);
  const xdd up[2] = {xdd_from_xint(xint_mul(u2, u)), xdd_from_xint(xint_sqr(u2))};
  window_horner_rev<CC, CZ>(P, P.b, u1, up, blocks != 0, -f, zr, zi, lo, hi, out[0], out[1], *rho, ct);
}

// bottom-up pass over [lo, hi]: out = (hr, hm), *rho = rho(hi), es = (E, S); returns ok
extern "C" int wc_rev(const double *b, int cc, int cz, const int32_t *k0, const int32_t *beta, const int32_t *delta,
                      const int64_t *rho0, const int32_t *first, int npieces, int log2_piece, double zr, double zi,
                      long long lo, long long hi, int blocks, double *out, long long *rho, float *es) {
  const DevPoly P = make_poly(b, cc, k0, beta, delta, rho0, first, npieces, log2_piece);
  Cert ct;
  if (cc && cz) rev<true, true>(P, zr, zi, lo, hi, blocks, out, rho, ct);
  else if (cc) rev<true, false>(P, zr, zi, lo, hi, blocks, out, rho, ct);
  else if (cz) rev<false, true>(P, zr, zi, lo, hi, blocks, out, rho, ct);
  else rev<false, false>(P, zr, zi, lo, hi, blocks, out, rho, ct);
  es[0] = ct.E;
  es[1] = ct.S;
  return ct.ok;
}

// the magnitude helpers: err_mag(x), mag_up(x), coef_mag_lo(x, y)
extern "C" void wc_mags(double x, double y, float *o) {
  o[0] = err_mag(x);
  o[1] = mag_up(x);
  o[2] = coef_mag_lo(x, y);
}

// one exact-multiplier step h w + b: out = (new hr, new hm), returns the step's error bound
extern "C" float wc_step_w(int cc, int cz, double hr, double hm, double wr, double wi, double br, double bi,
                           double *out) {
  float E = 0.0f, S = 0.0f;
  if (cc && cz) cstep_w<true, true>(hr, hm, wr, wi, br, bi, 0.0f, 1.0f, 1.0f, E, S);
  else if (cc) cstep_w<true, false>(hr, hm, wr, 0.0, br, bi, 0.0f, 1.0f, 1.0f, E, S);
  else if (cz) cstep_w<false, true>(hr, hm, wr, wi, br, 0.0, 0.0f, 1.0f, 1.0f, E, S);
  else cstep_w<false, false>(hr, hm, wr, 0.0, br, 0.0, 0.0f, 1.0f, 1.0f, E, S);
  out[0] = hr;
  out[1] = hm;
  return E;
}

// one double-double-multiplier step x v + b, v = (vhr + vlr) + i (vhi + vli)
extern "C" float wc_step_v(int cc, int cz, double xr, double xm, double vhr, double vlr, double vhi, double vli,
                           double br, double bi, double *out) {
  float E = 0.0f, S = 0.0f, Vu, Vd, Vl;
  if (cz) mult_bounds_dd<true>(vhr, vlr, vhi, vli, Vu, Vd, Vl);
  else mult_bounds_dd<false>(vhr, vlr, 0.0, 0.0, Vu, Vd, Vl);
  if (cc && cz) cstep_v<true, true>(xr, xm, vhr, vlr, vhi, vli, br, bi, 1.0f, 1.0f, Vl, 0.0f, 0.0f, E, S);
  else if (cc) cstep_v<true, false>(xr, xm, vhr, vlr, 0.0, 0.0, br, bi, 1.0f, 1.0f, Vl, 0.0f, 0.0f, E, S);
  else if (cz) cstep_v<false, true>(xr, xm, vhr, vlr, vhi, vli, br, 0.0, 1.0f, 1.0f, Vl, 0.0f, 0.0f, E, S);
  else cstep_v<false, false>(xr, xm, vhr, vlr, 0.0, 0.0, br, 0.0, 1.0f, 1.0f, Vl, 0.0f, 0.0f, E, S);
  out[0] = xr;
  out[1] = xm;
  return E;
}
