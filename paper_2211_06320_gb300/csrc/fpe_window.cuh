// FP64 window sums of Algorithm A_p (Q_lambda, eq. reducedQlambda) with their
// rounding-error certificates.  Host-compilable, so that a CPU test can run
// the same passes against exact rational sums.
//
// Each pass returns, beside its value, a Cert: E bounds the pass's FP64
// rounding error and S is a lower bound of its sum of term magnitudes, both
// at the pass's result scale in the units of the error bookkeeping
// (fpe_device.cuh: |computed - exact| <= 2^-53 2^-kMagOff E, S <=
// 2^kMagOff sum |terms|).  ok is false when a multiplier or a rescaling left
// the range that the bookkeeping covers.
#pragma once

#include "fpe_device.cuh"

#ifdef __CUDA_ARCH__
#define FPE_LDG(p) __ldg(p)
#else
#define FPE_LDG(p) (*(p))
#endif

namespace fpe {

struct Cert {
  float E, S, M;  // M >= 2^kMagOff |h|, the pass's result
  bool ok;
};

// Certificate threshold: a pass is accepted when E + M <= kCertC S.  M
// covers the rounding of the output to 53 bits (at most 2^-53 |P_w|, P_w
// the window sum, |P_w| <= sum of the passes' |h|); the fixed-point
// bookkeeping (below 2^-90 S) and the multiplier errors of the bottom-up
// pass (below L 2^-43 S, L <= 2^22) stay below 2^-20 S.  An accepted window
// value is then within 7.61 2^-53 S_w of the exact window sum: inside the
// 2^-50 S_w tolerance, and with the dropped terms (at most 2^(N - p - 3) <=
// 2^-55 S, §6) within 7.86 2^-53 S of P(z).
constexpr float kCertC = 7.6f;
// smallest multiplier modulus the bookkeeping accepts: above it, a
// subnormal component of w = 2^beta z, or of a double-double low part, errs
// by less than 2^-970 of |w|
constexpr float kCertMinMult = 0x1p-100f;
// largest |w| = |2^beta z| at which the bottom-up pass sums in blocks of four
// (with random-phase terms the blocks' certificates fail for under 3% of
// windows up to |w| = 2.25, for a quarter at 2.5)
constexpr float kBlockMaxW = 2.3f;

__host__ __device__ __forceinline__ bool cert_pass(const Cert &c) {
  return c.ok && add_up(c.E, c.M) <= mul_dn(c.S, kCertC);
}
__host__ __device__ __forceinline__ void cert_set(Cert &c, float E, float S, bool ok, double hr, double hm) {
  c.E = E;
  c.S = S;
  c.M = add_up(mag_up(hr), mag_up(hm));
  c.ok = ok;
}

// h <- h w + b (exact w) with its certificate terms; 4 FP64 FMA for complex z.
// bm: the coefficient's magnitude lower bound (DevPoly::bmag).
template <bool CC, bool CZ>
__host__ __device__ __forceinline__ void cstep_w(double &hr, double &hm, double wr, double wi, double br, double bi,
                                                 float bm, float Wu, float Wd, float &E, float &S) {
  float loc;
  if (CZ) {
    const double t1 = fma(-hm, wi, br), t2 = fma(hm, wr, bi);
    const double nr = fma(hr, wr, t1), ni = fma(hr, wi, t2);
    loc = add_up(add_up(err_mag(t1), err_mag(nr)), add_up(err_mag(t2), err_mag(ni)));
    hr = nr;
    hm = ni;
  } else {
    hr = fma(hr, wr, br);
    loc = err_mag(hr);
    if (CC) {
      hm = fma(hm, wr, bi);
      loc = add_up(loc, err_mag(hm));
    }
  }
  E = fma_up(E, Wu, loc);
  S = fma_dn(S, Wd, bm);
}

// bounds of |w| for w = wr + i wi (exact)
template <bool CZ>
__host__ __device__ __forceinline__ void mult_bounds(double wr, double wi, float &Wu, float &Wd) {
  Wu = CZ ? cabs_up(wr, wi) : fabs_up<0>(wr);
  Wd = CZ ? cabs_dn(wr, wi) : fabs_dn<0>(wr);
}

// scale a certificate by 2^d along with its value (|d| <= 120, else not covered)
__host__ __device__ __forceinline__ void cert_scale(float &E, float &S, bool &ok, int d) {
  ok = ok && d >= -120 && d <= 120;
  const float f = pow2f_bits(min(max(d, -120), 120));
  E = mul_up(E, f);
  S = mul_dn(S, f);
}

// x <- x v + (br + i bi) with v = (vhr + vlr) + i (vhi + vli) in double-double
// (8 FP64 FMA for complex z); the addend carries its own error bound Eb and
// magnitude Sb (a coefficient: 0 and |b|; a block sum: its certificate).
// The first two FMA of each component add a low-part product to a double,
// so each errs by at most that product (the double itself is a candidate of
// the rounding): together at most (|xr| + |xm|)(|vlr| + |vli|), which
// Vl = (|vlr| + |vli|) 2^53 (rounded up) turns into the scaled units.
template <bool CC, bool CZ>
__host__ __device__ __forceinline__ void cstep_v(double &xr, double &xm, double vhr, double vlr, double vhi,
                                                 double vli, double br, double bi, float Vu, float Vd, float Vl,
                                                 float Eb, float Sb, float &E, float &S) {
  const float lo = mul_up(add_up(mag_up(xr), mag_up(xm)), Vl);
  float loc;
  if (CZ) {
    const double r1 = fma(-xm, vli, br), q1 = fma(xm, vlr, bi);
    const double r2 = fma(xr, vlr, r1), q2 = fma(xr, vli, q1);
    const double r3 = fma(-xm, vhi, r2), q3 = fma(xm, vhr, q2);
    const double nr = fma(xr, vhr, r3), ni = fma(xr, vhi, q3);
    loc = add_up(add_up(lo, add_up(err_mag(r3), err_mag(nr))), add_up(err_mag(q3), err_mag(ni)));
    xr = nr;
    xm = ni;
  } else {
    const double r1 = fma(xr, vlr, br);
    const double nr = fma(xr, vhr, r1);
    loc = add_up(lo, err_mag(nr));
    if (CC) {
      const double q1 = fma(xm, vlr, bi);
      const double ni = fma(xm, vhr, q1);
      loc = add_up(loc, err_mag(ni));
      xm = ni;
    } else {
      xm = 0.0;
    }
    xr = nr;
  }
  E = fma_up(E, Vu, add_up(Eb, loc));
  S = fma_dn(S, Vd, Sb);
}

// bounds of a double-double multiplier's modulus, and Vl of cstep_v
template <bool CZ>
__host__ __device__ __forceinline__ void mult_bounds_dd(double hr, double lr, double hi, double li, float &Vu,
                                                        float &Vd, float &Vl) {
  if (CZ) {
    Vu = cabs_up_dd(hr, lr, hi, li);
    Vd = cabs_dn_dd(hr, lr, hi, li);
    Vl = add_up(fabs_up<53>(lr), fabs_up<53>(li));
  } else {
    Vu = add_up(fabs_up<0>(hr), fabs_up<0>(lr));
    Vd = fmaxf(fma_dn(-1.0f, fabs_up<0>(lr), fabs_dn<0>(hr)), 0.0f);
    Vl = fabs_up<53>(lr);
  }
}

// Horner over trimmed indices [lo, hi] on the rescaled coefficients b:
// returns h with sum_{k=lo}^{hi} b_k 2^rho(k) z^(k-lo) = h * 2^rho(lo).
// Piece j runs at w_j = 2^beta_j z; entering piece j from j+1 multiplies h by
// 2^delta_j (both exact).  Every term of a window has |h| <= L 2^(T + 66),
// so nothing overflows.
template <bool CC, bool CZ>
__host__ __device__ __forceinline__ void window_horner(const DevPoly &P, const double *__restrict__ b, double zr,
                                                       double zi, long long lo, long long hi, double &hr,
                                                       double &hm, long long &rho_lo, Cert &ct) {
  int j = P.piece_first[hi >> P.log2_piece];
  while (P.piece_k0[j + 1] <= hi) ++j;
  if (CC) {
    double2 c = reinterpret_cast<const double2 *>(b)[hi];
    hr = c.x;
    hm = c.y;
  } else {
    hr = b[hi];
    hm = 0.0;
  }
  const float *__restrict__ bmag = P.bmag;
  float E = 0.0f, S = FPE_LDG(&bmag[hi]);
  bool ok = true;
  long long k = hi - 1;
  long long k0 = max((long long)P.piece_k0[j], lo);
  while (true) {
    const int beta = P.piece_beta[j];
    const double wr = scale2(zr, beta);
    const double wi = CZ ? scale2(zi, beta) : 0.0;
    float Wu, Wd;
    mult_bounds<CZ>(wr, wi, Wu, Wd);
    ok = ok && Wd >= kCertMinMult;
    if (CC) {
      const double2 *b2 = reinterpret_cast<const double2 *>(b);
#pragma unroll 4
      for (; k >= k0; --k) {
        double2 c = FPE_LDG(&b2[k]);
        cstep_w<CC, CZ>(hr, hm, wr, wi, c.x, c.y, FPE_LDG(&bmag[k]), Wu, Wd, E, S);
      }
    } else {
#pragma unroll 4
      for (; k >= k0; --k) {
        double c = FPE_LDG(&b[k]);
        cstep_w<CC, CZ>(hr, hm, wr, wi, c, 0.0, FPE_LDG(&bmag[k]), Wu, Wd, E, S);
      }
    }
    if (k < lo) break;
    --j;  // k == piece_k0[j + 1] - 1: enter piece j
    const int dl = P.piece_delta[j];
    const double s = pow2i(dl);
    hr *= s;
    hm *= s;
    cert_scale(E, S, ok, dl);
    k0 = max((long long)P.piece_k0[j], lo);
  }
  rho_lo = P.piece_rho0[j] + (long long)P.piece_beta[j] * (lo - P.piece_k0[j]);
  cert_set(ct, E, S, ok, hr, hm);
}

// Blocks of B terms of the bottom-up pass, from k (the first index not yet
// summed) while a whole block fits in [k, kend].  With w = 1/v = 2^beta_j z
// (exact in FP64), B steps from K to K + B inside a piece are
//   h_{K+B} = v^B h_K + v^(B-1) s_K,  s_K = b_{K+1} + w (b_{K+2} + ... + w b_{K+B}),
// so G = w^(B-1) h obeys G_{K+B} = v^B G_K + s_K: the first block starts from
// G = v h_K + s_K, and h = v^(B-1) G at the end.  s_K is a top-down FP64
// Horner with the exact multiplier (B - 1 complex FMA steps, its rounding
// relative to the block's own terms) and the block step multiplies by v^B in
// double-double: 4 B + 4 FMA per B terms instead of 8 B.  uB = u^B and uB1 =
// u^(B-1) carry their own exponents; sh scales u to v on the piece.  The
// certificate follows the same recurrences: a block sum's bound is that of
// its exact-multiplier steps; the block steps and the final v^(B-1) add
// their own roundings.
template <bool CC, bool CZ, int B>
__host__ __device__ __forceinline__ void rev_blocks(const double *__restrict__ b, const float *__restrict__ bmag,
                                                    long long &k, long long kend, double wr, double wi, float Wu,
                                                    float Wd, double vhr, double vlr, double vhi, double vli,
                                                    float Vu, float Vd, float Vl, const xdd &uB, const xdd &uB1,
                                                    int sh, double &hr, double &hm, float &E, float &S, bool &ok) {
  auto load = [&](long long q, double &br, double &bi) {
    if (CC) {
      const double2 c = FPE_LDG(reinterpret_cast<const double2 *>(b) + q);
      br = c.x;
      bi = c.y;
    } else {
      br = FPE_LDG(b + q);
      bi = 0.0;
    }
  };
  const int sB = (int)uB.e + B * sh;
  const double ahr = scale2(uB.rh, sB), alr = scale2(uB.rl, sB);
  const double ahi = CZ ? scale2(uB.ih, sB) : 0.0, ali = CZ ? scale2(uB.il, sB) : 0.0;
  float Au, Ad, Al;
  mult_bounds_dd<CZ>(ahr, alr, ahi, ali, Au, Ad, Al);
  ok = ok && Wd >= kCertMinMult && Ad >= kCertMinMult;
  // s over [k0, k0 + B - 1] by top-down Horner with w, and its certificate
  auto block_sum = [&](long long k0, double &sr, double &si, float &Es, float &Ss) {
    load(k0 + B - 1, sr, si);
    Es = 0.0f;
    Ss = FPE_LDG(&bmag[k0 + B - 1]);
#pragma unroll
    for (int t = B - 2; t >= 0; --t) {
      double cr, ci;
      load(k0 + t, cr, ci);
      cstep_w<CC, CZ>(sr, si, wr, wi, cr, ci, FPE_LDG(&bmag[k0 + t]), Wu, Wd, Es, Ss);
    }
  };
  double sr, si;
  float Es, Ss;
  block_sum(k, sr, si, Es, Ss);
  cstep_v<CC, CZ>(hr, hm, vhr, vlr, vhi, vli, sr, si, Vu, Vd, Vl, Es, Ss, E, S);  // G = v h + s
  k += B;
  for (; k + B - 1 <= kend; k += B) {
    block_sum(k, sr, si, Es, Ss);
    cstep_v<CC, CZ>(hr, hm, ahr, alr, ahi, ali, sr, si, Au, Ad, Al, Es, Ss, E, S);  // G <- v^B G + s
  }
  // h = v^(B-1) G
  const int sC = (int)uB1.e + (B - 1) * sh;
  const double chr = scale2(uB1.rh, sC), clr = scale2(uB1.rl, sC);
  const double chi = CZ ? scale2(uB1.ih, sC) : 0.0, cli = CZ ? scale2(uB1.il, sC) : 0.0;
  float Cu, Cd, Cl;
  mult_bounds_dd<CZ>(chr, clr, chi, cli, Cu, Cd, Cl);
  (void)Cl;  // the low-part products below are rounded on their own, at their own tiny scale
  ok = ok && Cd >= kCertMinMult;
  float loc;
  double nr, ni;
  if (CZ) {
    const double r1 = -hm * cli, q1 = hm * clr;
    const double r2 = fma(hr, clr, r1), q2 = fma(hr, cli, q1);
    const double r3 = fma(-hm, chi, r2), q3 = fma(hm, chr, q2);
    nr = fma(hr, chr, r3);
    ni = fma(hr, chi, q3);
    loc = add_up(add_up(add_up(err_mag(r1), err_mag(r2)), add_up(err_mag(r3), err_mag(nr))),
                 add_up(add_up(err_mag(q1), err_mag(q2)), add_up(err_mag(q3), err_mag(ni))));
  } else {
    const double r1 = hr * clr;
    nr = fma(hr, chr, r1);
    loc = add_up(err_mag(r1), err_mag(nr));
    ni = 0.0;
    if (CC) {
      const double q1 = hm * clr;
      ni = fma(hm, chr, q1);
      loc = add_up(loc, add_up(err_mag(q1), err_mag(ni)));
    }
  }
  hr = nr;
  hm = ni;
  E = fma_up(E, Cu, loc);
  S = mul_dn(S, Cd);
}

// Bottom-up Horner over trimmed indices [lo, hi] with multiplier 1/z:
// returns h with sum_{k=lo}^{hi} b_k 2^rho(k) z^(k-hi) = h * 2^rho(hi).
// 1/z = u 2^ue with u in extended double-double (its powers up[0], up[1] =
// u^3, u^4 likewise, each with its own exponent).  Within piece j the
// step from k-1 to k multiplies by v_j = 2^-beta_j / z; crossing from piece
// j to j+1 first scales h by 2^-delta_j.  A single step is 8 FMA for complex
// z and coefficients (v in double-double).  With blocks set, runs of a piece
// go in blocks of four (rev_blocks) while |w| <= kBlockMaxW.  v and its powers are
// within 2^-96 of the exact ones (a reciprocal good to 2^-100, then a few
// 128-bit products), which the threshold kCertC allows for.
template <bool CC, bool CZ>
__host__ __device__ __forceinline__ void window_horner_rev(const DevPoly &P, const double *__restrict__ b,
                                                           const xdd &u, const xdd *up, bool blocks, int ue,
                                                           double zr, double zi, long long lo, long long hi,
                                                           double &hr, double &hm, long long &rho_hi, Cert &ct) {
  int j = P.piece_first[lo >> P.log2_piece];
  while (P.piece_k0[j + 1] <= lo) ++j;
  auto load = [&](long long k, double &br, double &bi) {
    if (CC) {
      const double2 c = FPE_LDG(reinterpret_cast<const double2 *>(b) + k);
      br = c.x;
      bi = c.y;
    } else {
      br = FPE_LDG(b + k);
      bi = 0.0;
    }
  };
  const float *__restrict__ bmag = P.bmag;
  load(lo, hr, hm);
  float E = 0.0f, S = FPE_LDG(&bmag[lo]);
  bool ok = true;
  long long k = lo + 1;
  while (k <= hi) {
    const int beta = P.piece_beta[j];
    const int sh = ue - beta;
    const int s1 = (int)u.e + sh;
    const double vhr = scale2(u.rh, s1), vlr = scale2(u.rl, s1);
    const double vhi = CZ ? scale2(u.ih, s1) : 0.0, vli = CZ ? scale2(u.il, s1) : 0.0;
    float Vu, Vd, Vl;
    mult_bounds_dd<CZ>(vhr, vlr, vhi, vli, Vu, Vd, Vl);
    ok = ok && Vd >= kCertMinMult;
    const long long kend = min((long long)P.piece_k0[j + 1] - 1, hi);
    if (blocks) {
      const double wr = scale2(zr, beta), wi = CZ ? scale2(zi, beta) : 0.0;
      float Wu, Wd;
      mult_bounds<CZ>(wr, wi, Wu, Wd);
      // blocks of four while |w| <= kBlockMaxW: beyond it the top term of a block,
      // rounded at each of the block sum's steps, costs more in the certificate
      // than the single steps' double-double roundings (8 FMA a term, not 5);
      // v^B and its low part stay normal for the shifts allowed
      if (kend - k + 1 >= 8 && sh > -200 && sh < 200 && Wu <= kBlockMaxW)
        rev_blocks<CC, CZ, 4>(b, bmag, k, kend, wr, wi, Wu, Wd, vhr, vlr, vhi, vli, Vu, Vd, Vl, up[1], up[0], sh,
                              hr, hm, E, S, ok);
    }
    for (; k <= kend; ++k) {
      double br, bi;
      load(k, br, bi);
      cstep_v<CC, CZ>(hr, hm, vhr, vlr, vhi, vli, br, bi, Vu, Vd, Vl, 0.0f, FPE_LDG(&bmag[k]), E, S);
    }
    if (k > hi) break;
    // k is the first index of piece j + 1: rescale, one step with v_j, move on
    const int dl = -P.piece_delta[j];
    const double s2 = pow2i(dl);
    hr *= s2;
    hm *= s2;
    cert_scale(E, S, ok, dl);
    double br, bi;
    load(k, br, bi);
    cstep_v<CC, CZ>(hr, hm, vhr, vlr, vhi, vli, br, bi, Vu, Vd, Vl, 0.0f, FPE_LDG(&bmag[k]), E, S);
    ++k;
    ++j;
  }
  rho_hi = P.piece_rho0[j] + (long long)P.piece_beta[j] * (hi - P.piece_k0[j]);
  cert_set(ct, E, S, ok, hr, hm);
}

}  // namespace fpe
