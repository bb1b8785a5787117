// Host model of one tile of the tensor-core window sums: the same fixed-point
// steps as k_tc_tau, k_tc_pre, k_tc_sum and k_tc_finalize (fpe_tc.cu), with
// the MMAs replaced by exact integer dot products of the same digits (the
// tensor core's fp32 sums are exact, which tests/test_tc_arith_host.py
// checks), on one piece with k0 = 0, beta = 0, rho = 0, no valuation.  The
// result per point is sum_{k = 32 mlo}^{32 (mlo + nblk) - 1} b_k z^k as an
// xint; tests/test_tc_model_host.py compares it with a high-precision sum.
#include <climits>
#include <cmath>

#include "fpe_tc_arith.cuh"
using namespace fpe;

namespace {

constexpr int kSub = 8;

xint pow_x(xint b, long long n) {  // b^n, n >= 1, by binary powering (as the kernel)
  xint r = b;
  bool have = false;
  for (; n > 0; n >>= 1) {
    if (n & 1) {
      r = have ? xint_mul(r, b) : b;
      have = true;
    }
    if (n > 1) b = xint_sqr(b);
  }
  return r;
}

constexpr int kFold = 16;  // sub-tiles between the 128-bit folds of a thread's Horner value

constexpr int kPer = 4;  // threads per point, each taking blocks 2 h, 2 h + 1 of a sub-tile of 8

struct Point {
  int sd_re[kTB][kSl], sd_im[kTB][kSl];  // signed Z' digits of u^i
  int eq;                                // Z' = F 2^(eq - 70)
  xint W[4];
  xh w1, w8;
  xint wf;  // W^(8 kFold)
};

void digits(u128 F, int neg, int (&d)[kSl]) {
  uint32_t x[kSl];
  bchunks70(F, x);
  const DigitSign s = digit_sign((uint32_t)neg);
  for (int j = 0; j < kSl; ++j) d[j] = (int)fmaf(tc_bitsf(x[j]), s.s, s.k);
}

}  // namespace

// b: 2 * 32 * nblk doubles (re, im) for k = 32 mlo ...; points (zr, zi); tilt exponent c;
// chunk: blocks per work item (a multiple of 8).  Out per point: X lo, X hi, Y lo, Y hi, sx, sy, e.
extern "C" void t_tile(const double *b, long long mlo, long long nblk, const double *zr, const double *zi, int npts,
                       double c, long long chunk, unsigned long long *ox, int *os, long long *oe) {
  // k_tc_tau
  const double tau = exp2(c);
  int tf = 0;
  frexp(tau, &tf);
  const double tmant = ldexp(tau, -tf);
  unsigned long long tm[kTB];
  int te[kTB];
  for (int i = 0; i < kTB; ++i) {
    xint ti = xint_norm((u128)1 << 126, 0, 0, 0, 0);
    if (i > 0) {
      ti = xint_pow_unit(tmant, 0.0, i);
      ti.e += (long long)tf * i;
    }
    tm[i] = (unsigned long long)(ti.x >> 63);
    te[i] = (int)(ti.e - 63);
  }
  xint inv = recip_xint(tmant, 0.0);
  inv.e -= tf;
  xint t32 = xint_pow_unit(tmant, 0.0, kTB);
  t32.e += (long long)tf * kTB;

  // k_tc_pre
  Point *pts = new Point[npts];
  for (int p = 0; p < npts; ++p) {
    Point &P = pts[p];
    const xint u = xint_mul(xint_from_dd2(zr[p], 0.0, zi[p], 0.0, 0), inv);
    const xh uh = xh_from_xint(u);
    const float mx = (float)(unsigned long long)(u.x >> 64) * 0x1p-62f;
    const float my = (float)(unsigned long long)(u.y >> 64) * 0x1p-62f;
    const float l = 0.5f * log2f(fmaf(mx, mx, my * my)) + (float)u.e;
    const int eQ = std::max(0, (int)ceilf(31.0f * l + 1e-3f)) + 1;
    xh cur = xh_norm(1ull << 63, 0, 0, 0, 0);
    for (int i = 0; i < kTB; ++i) {
      if (i > 0) cur = xh_mul(cur, uh);
      const int sr = eQ + 1 + 63 - 70 - (int)cur.e;
      digits(shift_to70((u128)cur.x, sr), cur.sx, P.sd_re[i]);
      digits(shift_to70((u128)cur.y, sr), cur.sy, P.sd_im[i]);
    }
    xint u32 = u;
    for (int k = 0; k < 5; ++k) u32 = xint_sqr(u32);
    P.W[0] = xint_mul(u32, t32);
    for (int k = 1; k < 4; ++k) P.W[k] = xint_sqr(P.W[k - 1]);
    P.wf = P.W[3];
    for (int q = 1; (1 << q) <= kFold; ++q) P.wf = xint_sqr(P.wf);
    P.eq = eQ + 1;
    P.w1 = xh_from_xint(P.W[0]);
    P.w8 = xh_from_xint(P.W[3]);
  }

  // k_tc_sum, one work item at a time: per point four threads h = 0..3, each
  // taking blocks 2 h, 2 h + 1 of every sub-tile of 8, from the top down, by
  // H <- H W^8 + C_1 W + C_0 in 64-bit mantissas, folded into a 128-bit value
  // every kFold sub-tiles; V = A_0 + W^2 (A_1 + W^2 (A_2 + W^2 A_3))
  const long long nit = (nblk + chunk - 1) / chunk;
  xint *slot = new xint[nit * npts];
  const xint zero0 = xint_norm(0, 0, 0, 0, 0);
  for (long long it = 0; it < nit; ++it) {
    const long long mb = mlo + it * chunk, me = std::min(mlo + nblk, mb + chunk);
    const int nsub = (int)((me - mb + kSub - 1) / kSub);
    xh *H = new xh[npts * kPer];
    xint *A = new xint[npts * kPer];
    xh *Cb = new xh[npts * kSub];  // the current sub-tile's block values
    for (int q = 0; q < npts * kPer; ++q) {
      H[q] = xh_norm(0, 0, 0, 0, 0);
      A[q] = zero0;
    }
    for (int ts = nsub - 1; ts >= 0; --ts) {
      const long long m0 = mb + (long long)kSub * ts;
      for (int g = kSub - 1; g >= 0; --g) {
        const long long m = m0 + g;
        // A' digits of block m: lane i = term k = 32 m + i
        int ad_re[kTB][kSl], ad_im[kTB][kSl];
        u128 pr[kTB], pi[kTB];
        int er_[kTB], ei_[kTB], top = INT_MIN;
        double brs[kTB], bis[kTB];
        for (int i = 0; i < kTB; ++i) {
          const bool in = m < me;
          const double br = in ? b[2 * (32 * (m - mlo) + i)] : 0.0, bi = in ? b[2 * (32 * (m - mlo) + i) + 1] : 0.0;
          brs[i] = br;
          bis[i] = bi;
          pr[i] = pi[i] = 0;
          er_[i] = ei_[i] = 0;
          auto prod = [&](double x, u128 &pp, int &E) {
            unsigned long long bits;
            memcpy(&bits, &x, 8);
            bits &= 0x7fffffffffffffffull;
            if (bits == 0) return;
            const int ex = (int)(bits >> 52);
            const unsigned long long mm = ex ? ((bits & 0xfffffffffffffull) | 0x10000000000000ull)
                                             : (bits & 0xfffffffffffffull);
            pp = (u128)mm * tm[i];
            E = (ex ? ex : 1) - 1075 + te[i];
            top = std::max(top, 127 - clz128(pp) + E);
          };
          prod(br, pr[i], er_[i]);
          prod(bi, pi[i], ei_[i]);
        }
        const int eR = top == INT_MIN ? 0 : top + 2;
        for (int i = 0; i < kTB; ++i) {
          digits(pr[i] ? shift_to70(pr[i], eR - 70 - er_[i]) : (u128)0, brs[i] < 0.0, ad_re[i]);
          digits(pi[i] ? shift_to70(pi[i], eR - 70 - ei_[i]) : (u128)0, bis[i] < 0.0, ad_im[i]);
        }
        for (int p = 0; p < npts; ++p) {
          const Point &P = pts[p];
          // out_re = sum_i A'_re Z'_re - A'_im Z'_im, out_im = sum_i A'_im Z'_re + A'_re Z'_im, per digit pair
          float acc_re[kAcc], acc_im[kAcc];
          for (int t = 0; t < kAcc; ++t) {
            long long sre = 0, sim = 0;
            for (int s = 0; s <= t; ++s) {
              if (s >= kSl || t - s >= kSl) continue;
              for (int i = 0; i < kTB; ++i) {
                sre += (long long)ad_re[i][s] * P.sd_re[i][t - s] - (long long)ad_im[i][s] * P.sd_im[i][t - s];
                sim += (long long)ad_im[i][s] * P.sd_re[i][t - s] + (long long)ad_re[i][s] * P.sd_im[i][t - s];
              }
            }
            acc_re[t] = (float)sre;  // exact: below 2^22
            acc_im[t] = (float)sim;
          }
          xh C = xh_norm(0, 0, 0, 0, 0);
          if (m < me) {
            u128 xr, xi;
            int sr, si;
            join_vals(acc_re, xr, sr);
            join_vals(acc_im, xi, si);
            C = xh_from128(xr, sr, xi, si, 49 + (long long)eR + P.eq);
          }
          Cb[p * kSub + g] = C;
        }
      }
      for (int p = 0; p < npts; ++p)
        for (int hh = 0; hh < kPer; ++hh) {
          xh &h = H[p * kPer + hh];
          xh T1 = Cb[p * kSub + 2 * hh + 1];
          if (T1.x || T1.y) T1 = xh_mul(T1, pts[p].w1);
          if (h.x || h.y) h = xh_mul(h, pts[p].w8);
          h = xh_add(xh_add(h, T1), Cb[p * kSub + 2 * hh]);
          if (ts % kFold == 0) {  // fold
            xint &a = A[p * kPer + hh];
            if (a.x || a.y) a = xint_mul(a, pts[p].wf);
            a = xint_add(a, xint_from_xh(h));
            h = xh_norm(0, 0, 0, 0, 0);
          }
        }
    }
    for (int p = 0; p < npts; ++p) {  // V = A_0 + W^2 (A_1 + W^2 (A_2 + W^2 A_3)), A_1..3 passed in 64 bits
      xint V = xint_from_xh(xh_from_xint(A[p * kPer + kPer - 1]));
      for (int q = kPer - 2; q >= 0; --q) {
        if (V.x || V.y) V = xint_mul(V, pts[p].W[1]);
        V = xint_add(V, q > 0 ? xint_from_xh(xh_from_xint(A[p * kPer + q])) : A[p * kPer]);
      }
      slot[it * npts + p] = V;
    }
    delete[] H;
    delete[] A;
    delete[] Cb;
  }

  // k_tc_finalize: one thread per point up to 4 items, else 3 item threads + a butterfly over 4
  const xint zero = xint_norm(0, 0, 0, 0, 0);
  for (int p = 0; p < npts; ++p) {
    const int L = nit <= 4 ? 1 : 4, nh = L > 1 ? L - 1 : 1;
    const long long per = (nit + nh - 1) / nh;
    const xint Wc = nit > 1 ? pow_x(pts[p].W[3], chunk / 8) : zero;
    xint part[8];
    for (int q = 0; q < L; ++q) {
      const long long c0 = q * per, c1 = q < nh ? std::min(nit, c0 + per) : c0;
      xint V = zero;
      for (long long cc = c1 - 1; cc >= c0; --cc) {
        if (V.x || V.y) V = xint_mul(V, Wc);
        V = xint_add(V, slot[cc * npts + p]);
      }
      if (c0 > 0 && c0 < c1 && (V.x || V.y)) V = xint_mul(V, pow_x(Wc, c0));
      part[q] = V;
    }
    for (int o = 1; o < L; o <<= 1) {
      xint nxt[8];
      for (int q = 0; q < L; ++q) nxt[q] = xint_add(part[q], part[q ^ o]);
      for (int q = 0; q < L; ++q) part[q] = nxt[q];
    }
    int f = 0;
    frexp(fabs(zr[p]) > fabs(zi[p]) ? zr[p] : zi[p], &f);
    const xint zp = xint_pow_z(zr[p], zi[p], 32 * mlo, f);
    xint V = part[0];
    if (V.x || V.y) V = xint_mul(V, zp);
    ox[4 * p] = (unsigned long long)V.x;
    ox[4 * p + 1] = (unsigned long long)(V.x >> 64);
    ox[4 * p + 2] = (unsigned long long)V.y;
    ox[4 * p + 3] = (unsigned long long)(V.y >> 64);
    os[2 * p] = V.sx;
    os[2 * p + 1] = V.sy;
    oe[p] = V.e;
  }
  delete[] slot;
  delete[] pts;
}
