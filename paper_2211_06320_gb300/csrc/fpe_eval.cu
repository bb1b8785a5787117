// Evaluation phase of Algorithm A_p (its evaluation part, §5.2) on the GPU.
//
// Stages, all asynchronous on the caller's stream, with grid sizes that depend
// only on n (so the sequence can be captured in a CUDA graph):
//   k_locate    per point: lambda = log2|z|, k_lambda and N by binary search on
//               the cover's slopes (eq. defN), l and r by two binary searches
//               (def. LRN); bucket key from lambda; histogram.
//   k_scan_bins exclusive scan of the bucket histogram (one block).
//   k_scatter   points to bucketed order (points of similar |z| together, so a
//               warp's lanes get windows of similar length and position);
//               long windows listed separately.
//   k_sums      all window sums in one persistent launch: warps take work
//               items from a counter, first the warp groups of long windows
//               (32 lane chunks of one window), then 32 bucketed points each
//               (one thread per short window); the last group of a long
//               window combines its groups and applies z^(l + v).
//
// Summation order.  The terms of a window peak at k_lambda.  Horner's scheme
// is accurate when each step adds a term no smaller than the ones already
// summed, so the window is summed in two parts that both move toward the
// peak: [k_lambda, r] top-down with multiplier z (4 FMA per complex term),
// and [l, k_lambda - 1] bottom-up with multiplier 1/z held in double-double,
// in blocks of four (20 FMA per four terms, see window_horner_rev).
// Top-down over the whole window (the paper's z^l times Horner) rounds a
// partial sum already as large as P(z) at every one of the ~T/lambda steps
// below the peak, which in FP64 exceeds 2^-50 S(z).  FPE_ACCURATE sums
// top-down on the integer pipe in 128-bit fixed point instead, and so does
// the default mode for the lane chunks of long windows and for every window
// of real points with real coefficients: on this GPU (FP64 at about 1.7 FMA
// per cycle per SM) the integer pipe sums those faster than the FP64 passes
// with their certificates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "fpe_device.cuh"
#include "fpe_internal.h"
#include "fpe_window.cuh"

namespace fpe {

// ---------------------------------------------------------------------------
// location (Alg. A_p: k_lambda, N, l, r; eq. defN, def. LRN)
// ---------------------------------------------------------------------------

struct Window {
  long long lo, hi;  // trimmed
  long long kl;      // trimmed k_lambda
  double N;          // trimmed maximum
  double lam;
  int flags;
};

template <bool CZ>
__device__ __forceinline__ Window locate_point(const DevPoly &P, double zr, double zi) {
  Window w;
  w.lo = 1;
  w.hi = 0;
  w.kl = 0;
  w.N = 0.0;
  w.lam = 0.0;
  w.flags = 0;
  if (!isfinite(zr) || (CZ && !isfinite(zi))) {
    w.flags = kPointNonFinite;
    return w;
  }
  if (zr == 0.0 && (!CZ || zi == 0.0)) {
    w.flags = kPointZero;
    return w;
  }
  double lam;
  if (CZ) {
    // lambda = log2|z| = f + log2|z 2^-f| with |z 2^-f| in [0.5, sqrt 2)
    int f = frexp_exp(fmax(fabs(zr), fabs(zi)));
    double xr = scale2(zr, -f), xi = scale2(zi, -f);
    lam = (double)f + 0.5 * log2(fma(xr, xr, xi * xi));
  } else {
    lam = log2(fabs(zr));
  }
  w.lam = lam;
  const int nh = P.n_hull;
  const double *hk = P.hull_k, *hs = P.hull_s, *sg = P.hull_sig;
  // k_lambda: first vertex whose right segment has slope <= -lambda (ties: leftmost)
  int a = 0, b = nh - 1;
  while (a < b) {
    int m = (a + b) >> 1;
    if (sg[m] <= -lam)
      b = m;
    else
      a = m + 1;
  }
  const int is = a;
  const double N = fma(lam, hk[is], hs[is]);
  const double thr = N - P.T;
  // left branch: cover + lambda Id increases on vertices [0, is]
  long long lo;
  if (is == 0 || fma(lam, hk[0], hs[0]) >= thr) {
    lo = (long long)hk[0];
  } else {
    int x = 0, y = is;  // f(x) < thr <= f(y)
    while (y - x > 1) {
      int m = (x + y) >> 1;
      if (fma(lam, hk[m], hs[m]) < thr)
        x = m;
      else
        y = m;
    }
    double fx = fma(lam, hk[x], hs[x]);
    double t = hk[x] + (thr - fx) / (sg[x] + lam);
    lo = (long long)ceil(t);
    lo = max(lo, (long long)hk[x] + 1);
    lo = min(lo, (long long)hk[x + 1]);
  }
  // right branch: decreases on vertices [is, nh - 1]
  long long hi;
  if (is == nh - 1 || fma(lam, hk[nh - 1], hs[nh - 1]) >= thr) {
    hi = (long long)hk[nh - 1];
  } else {
    int x = is, y = nh - 1;  // f(x) >= thr > f(y)
    while (y - x > 1) {
      int m = (x + y) >> 1;
      if (fma(lam, hk[m], hs[m]) < thr)
        y = m;
      else
        x = m;
    }
    double fx = fma(lam, hk[x], hs[x]);
    double t = hk[x] + (thr - fx) / (sg[x] + lam);
    hi = (long long)floor(t);
    hi = max(hi, (long long)hk[x]);
    hi = min(hi, (long long)hk[y] - 1);
  }
  w.lo = lo;
  w.hi = hi;
  w.kl = (long long)hk[is];
  w.N = N;
  return w;
}

__device__ __forceinline__ uint32_t bucket_of(double lam, int flags) {
  if (flags) return 0;
  // monotone squashing of lambda onto [0, 1): atan(lambda / 4) / pi + 1/2
  float t = atanf((float)lam * 0.25f) * 0.318309886f + 0.5f;
  int b = (int)(t * (float)kNumBins);
  return (uint32_t)min(max(b, 0), kNumBins - 1);
}

// Bucket of a point whose window [lo, hi] (trimmed) qualifies for the
// tensor-core sums: at least tc_min_window terms inside one tensor-core piece
// r.  Bins kNumBins + r kTcBinsPerPiece + [0, kTcBinsPerPiece) order mu =
// lambda + beta logarithmically (kTcBinsPerBinade bins per binade of |mu|
// over [2^-24, 2^8], negative mu first), so consecutive points share windows.
__device__ __forceinline__ bool tc_bucket(const DevPoly &P, long long lo, long long hi, double lam,
                                          long long tc_min_window, uint32_t &key) {
  if (hi - lo + 1 < tc_min_window) return false;
  int j = P.piece_first[lo >> P.log2_piece];
  while (P.piece_k0[j + 1] <= lo) ++j;
  if (P.piece_k0[j + 1] <= hi) return false;
  int r = -1;
  for (int q = 0; q < P.n_tc && q < kTcMaxPieces; ++q)
    if (P.tc_piece[q] == j) r = q;
  if (r < 0) return false;
  const double mu = lam + (double)P.piece_beta[j];
  const float a = (float)fabs(mu);
  int h = 0;
  if (a >= 0x1p-24f) h = min((int)((log2f(a) + 24.0f) * (float)kTcBinsPerBinade), kTcBinsPerPiece / 2 - 1);
  const int b = mu < 0.0 ? kTcBinsPerPiece / 2 - 1 - h : kTcBinsPerPiece / 2 + h;
  key = (uint32_t)(kNumBins + r * kTcBinsPerPiece + b);
  return true;
}

template <bool CZ>
__global__ void k_locate(DevPoly P, int n, const double *__restrict__ zre, const double *__restrict__ zim,
                         long long *__restrict__ lo_out, long long *__restrict__ hi_out,
                         long long *__restrict__ kl_out, double *__restrict__ N_out, uint32_t *__restrict__ key,
                         uint32_t *__restrict__ rank, uint32_t *__restrict__ hist, long long tc_min_window) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double zr = zre[p], zi = CZ ? zim[p] : 0.0;
  Window w = locate_point<CZ>(P, zr, zi);
  lo_out[p] = w.lo + (w.flags ? 0 : P.v);
  hi_out[p] = w.hi + (w.flags ? 0 : P.v);
  kl_out[p] = w.kl;
  N_out[p] = w.flags ? 0.0 : w.N + w.lam * (double)P.v;
  uint32_t k = bucket_of(w.lam, w.flags);
  if (tc_min_window > 0 && !w.flags) tc_bucket(P, w.lo, w.hi, w.lam, tc_min_window, k);
  key[p] = k;
  rank[p] = atomicAdd(&hist[k], 1u);  // the point's place within its bin
}

// Exclusive scan of the nbins-word histogram (nbins a multiple of
// kScanTile) into cursors, in two launches of one 256-thread block per tile
// of kScanTile bins (coalesced 16-byte loads): k_scan_tiles writes each
// tile's total after the counters, k_scan_bins adds the totals of the tiles
// before its own to a scan of the tile.  k_scan_bins also resets the
// counters and records where each tensor-core piece's points start in
// bucketed order (a piece's first bin starts a tile).
constexpr int kScanTile = 1024;
static_assert(kNumBins % kScanTile == 0 && kTcBinsPerPiece % kScanTile == 0, "tiles of whole bins");

__device__ __forceinline__ uint32_t block_sum256(uint32_t v, uint32_t *red) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) tot += red[i];
  return tot;
}

__global__ void __launch_bounds__(256) k_scan_tiles(uint32_t *bins, int nbins) {
  __shared__ uint32_t red[8];
  const uint4 v = reinterpret_cast<const uint4 *>(bins + (size_t)blockIdx.x * kScanTile)[threadIdx.x];
  const uint32_t tot = block_sum256(v.x + v.y + v.z + v.w, red);
  if (threadIdx.x == 0) bins[2 * nbins + kNumCounters + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_scan_bins(uint32_t *bins, int nbins) {
  __shared__ uint32_t red[8], wsum[8];
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int ntiles = nbins / kScanTile;
  uint32_t *cnt = bins + 2 * nbins;
  const uint32_t *tile_tot = cnt + kNumCounters;
  uint32_t part = 0;  // the tiles before this one
  for (int i = t; i < b; i += 256) part += tile_tot[i];
  const uint32_t off = block_sum256(part, red);
  const uint4 v = reinterpret_cast<const uint4 *>(bins + (size_t)b * kScanTile)[t];
  const uint32_t own = v.x + v.y + v.z + v.w;
  uint32_t inc = own;  // inclusive scan of the threads' sums within the warp
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  uint32_t before = 0;  // the warps before this one
  for (int i = 0; i < wid; ++i) before += wsum[i];
  uint4 o4;
  o4.x = off + before + inc - own;
  o4.y = o4.x + v.x;
  o4.z = o4.y + v.y;
  o4.w = o4.z + v.z;
  reinterpret_cast<uint4 *>(bins + nbins + (size_t)b * kScanTile)[t] = o4;
  // counters: reset by block 0, except the tensor-core piece starts, which the
  // block holding the piece's first bin writes (the last block: pieces
  // without bins, and the total)
  if (b == 0 && t < kNumCounters && (t < kCntTcStart || t > kCntTcStart + kTcMaxPieces)) cnt[t] = 0;
  if (t <= kTcMaxPieces) {
    const int first = kNumBins + t * kTcBinsPerPiece;
    if (t < kTcMaxPieces && first < nbins) {
      if (first == b * kScanTile) cnt[kCntTcStart + t] = off;
    } else if (b == ntiles - 1) {
      uint32_t tot = 0;
      for (int i = 0; i < 8; ++i) tot += wsum[i];
      cnt[kCntTcStart + t] = off + tot;
    }
  }
}

static void launch_scan_bins(uint32_t *bins, int nbins, cudaStream_t st) {
  k_scan_tiles<<<nbins / kScanTile, 256, 0, st>>>(bins, nbins);
  k_scan_bins<<<nbins / kScanTile, 256, 0, st>>>(bins, nbins);
}

template <bool CZ>
__global__ void k_scatter(DevPoly P, int n, const double *__restrict__ zre, const double *__restrict__ zim,
                          const long long *__restrict__ lo, const long long *__restrict__ hi,
                          const long long *__restrict__ kl, const double *__restrict__ N,
                          const uint32_t *__restrict__ key, const uint32_t *__restrict__ rank, uint32_t *bins,
                          PointRec *__restrict__ rec, int32_t *__restrict__ long_list,
                          int32_t *__restrict__ long_ngroups, int32_t *__restrict__ long_gbase,
                          int32_t *__restrict__ extra_owner, int32_t *__restrict__ extra_group, int extra_cap,
                          int32_t *status, long long long_window, long long span, int nbins) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t kp = key[p];
  const uint32_t pos = bins[nbins + kp] + rank[p];  // bin start (scanned) + place in the bin
  PointRec r;
  r.zr = zre[p];
  r.zi = CZ ? zim[p] : 0.0;
  long long l = lo[p], h = hi[p];
  r.flags = 0;
  if (!isfinite(r.zr) || !isfinite(r.zi)) {
    r.flags = kPointNonFinite;
    atomicOr(status, kStatusNonFinite);
  } else if (r.zr == 0.0 && r.zi == 0.0) {
    r.flags = kPointZero;
  }
  r.lo = r.flags ? 1 : l - P.v;
  r.hi = r.flags ? 0 : h - P.v;
  r.kl = kl[p];
  r.N = N[p];
  r.orig = p;
  r.pid = 0;
  r.pad = 0;
  if (!r.flags && kp >= (uint32_t)kNumBins) r.flags = kPointTC;  // summed by the tensor-core kernels
  rec[pos] = r;
  if (!r.flags && r.hi - r.lo + 1 > long_window)
    list_long_window(r.hi - r.lo + 1, span, pos, bins + 2 * nbins, long_list, long_ngroups, long_gbase,
                     extra_owner, extra_group, extra_cap);
}

// ---------------------------------------------------------------------------
// window sums (Alg. A_p: Q_lambda, eq. reducedQlambda)
// ---------------------------------------------------------------------------

__device__ __forceinline__ fpe_xc64 special_value(const DevPoly &P, int flags) {
  fpe_xc64 o;
  if (flags & kPointNonFinite) {
    o.re = __longlong_as_double(0x7ff8000000000000ll);
    o.im = o.re;
    o.e = 0;
  } else {  // z = 0: P(0) = a_0 (0 when the valuation is positive)
    o.re = P.a0_re;
    o.im = P.a0_im;
    o.e = (P.a0_re == 0.0 && P.a0_im == 0.0) ? 0 : P.a0_e;
  }
  return o;
}

__device__ __forceinline__ void write_diag(const DevPoly &P, const PointRec &r, const fpe_xc64 &o,
                                           int32_t *nterms, int32_t *bits_lost) {
  if (nterms) nterms[r.orig] = r.flags ? (r.flags == kPointZero ? (P.v == 0 ? 1 : 0) : 0)
                                       : P.gcount[r.hi + 1] - P.gcount[r.lo];
  if (bits_lost) {
    int bl = 0;
    if (!r.flags && (o.re != 0.0 || o.im != 0.0)) {
      double c = ceil(r.N) - (double)o.e;
      bl = c > 0.0 ? (int)fmin(c, 2.0e9) : 0;
    }
    bits_lost[r.orig] = bl;
  }
}

// sum_{k=lo}^{hi} a_k z^(k - base) in extended double-double for a range on
// either side of the peak kl or straddling it.  The part at or above kl is
// summed top-down (relative to z^max(kl, lo)), the part below bottom-up
// (relative to z^(its top index)); base is kl - 1 when both parts exist.
// ok: both parts passed their rounding-error certificates (cert_pass); the
// caller sums the range again on the integer pipe when it is false.
template <bool CC, bool CZ>
__device__ __forceinline__ xint range_sum(const DevPoly &P, double zr, double zi, double mr, double mi, int f,
                                          const xint &u, long long lo, long long hi, long long kl, long long &base,
                                          bool &ok) {
  constexpr long long kBlockMin = 16;  // below-peak terms from which the blocked pass pays for u^3, u^4
  xint X = xint_norm(0, 0, 0, 0, 0);
  const long long top_lo = max(kl, lo);
  const long long low_hi = min(top_lo - 1, hi);
  const bool has_up = top_lo <= hi, has_low = lo <= low_hi;
  ok = true;
  if (has_up) {
    double hr, hm;
    long long rho;
    Cert ct;
    window_horner<CC, CZ>(P, P.b, zr, zi, top_lo, hi, hr, hm, rho, ct);
    ok = cert_pass(ct);
    X = xint_from_dd2(hr, 0.0, hm, 0.0, rho);
    base = top_lo;
  }
  if (has_low) {
    double hr, hm;
    long long rho;
    const bool blocks = low_hi - lo + 1 >= kBlockMin;
    const xdd u1 = xdd_from_xint(u);
    xdd up[2] = {u1, u1};
    if (blocks) {  // powers u^3, u^4 of 1/m on the integer pipe
      const xint u2 = xint_sqr(u);
      up[0] = xdd_from_xint(xint_mul(u2, u));
      up[1] = xdd_from_xint(xint_sqr(u2));
    }
    Cert ct;
    window_horner_rev<CC, CZ>(P, P.b, u1, up, blocks, -f, zr, zi, lo, low_hi, hr, hm, rho, ct);
    ok = ok && cert_pass(ct);
    if (has_up && (X.x || X.y)) X = xint_mul(X, xint_from_dd2(mr, 0.0, mi, 0.0, f));  // z^top_lo = z * z^low_hi
    X = xint_add(X, xint_from_dd2(hr, 0.0, hm, 0.0, rho));
    base = low_hi;
  }
  return X;
}

// ---------------------------------------------------------------------------
// FP32 mode (FPE_FP32, p <= 24): coefficients rounded to FP32 on 32-term
// pieces, Horner on the FP32 pipe.  The multiplier (2^beta z top-down,
// 2^-beta / z bottom-up) is a float-float pair: an FP32-rounded multiplier
// would put a relative error L 2^-24 on the L-th power, while 48 bits keep
// it below 2^-28 for L <= 2^20.  8 FP32 FMA per complex term.
// ---------------------------------------------------------------------------
struct ff2 {
  float rh, rl, ih, il;
};
__device__ __forceinline__ ff2 ff_split(double r, double i) {
  const float rh = __double2float_rn(r), ih = __double2float_rn(i);
  return {rh, __double2float_rn(r - (double)rh), ih, __double2float_rn(i - (double)ih)};
}
// 2^k as a float, k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

template <bool CC, bool CZ>
__device__ __forceinline__ void ff_step(float &hr, float &hm, const ff2 &w, float br, float bi) {
  if (CZ) {
    const float nr = fmaf(hr, w.rh, fmaf(-hm, w.ih, fmaf(hr, w.rl, fmaf(-hm, w.il, br))));
    const float ni = fmaf(hr, w.ih, fmaf(hm, w.rh, fmaf(hr, w.il, fmaf(hm, w.rl, bi))));
    hr = nr;
    hm = ni;
  } else {
    hr = fmaf(hr, w.rh, fmaf(hr, w.rl, br));
    if (CC) hm = fmaf(hm, w.rh, fmaf(hm, w.rl, bi));
  }
}

template <bool CC>
__device__ __forceinline__ void load_bf(const float *__restrict__ b, long long k, float &br, float &bi) {
  if (CC) {
    const float2 c = __ldg(reinterpret_cast<const float2 *>(b) + k);
    br = c.x;
    bi = c.y;
  } else {
    br = __ldg(b + k);
    bi = 0.0f;
  }
}

// top-down over [lo, hi]: sum b_k 2^rho(k) z^(k-lo) = h 2^rho(lo)
template <bool CC, bool CZ>
__device__ __forceinline__ void window_horner_f32(const DevPoly &P, double zr, double zi, long long lo,
                                                  long long hi, float &hr, float &hm, long long &rho_lo) {
  const float *__restrict__ b = P.bf;
  int j = P.piece_first[hi >> P.log2_piece];
  while (P.piece_k0[j + 1] <= hi) ++j;
  load_bf<CC>(b, hi, hr, hm);
  long long k = hi - 1;
  long long k0 = max((long long)P.piece_k0[j], lo);
  while (true) {
    const int beta = P.piece_beta[j];
    const ff2 w = ff_split(scale2(zr, beta), CZ ? scale2(zi, beta) : 0.0);
#pragma unroll 4
    for (; k >= k0; --k) {
      float br, bi;
      load_bf<CC>(b, k, br, bi);
      ff_step<CC, CZ>(hr, hm, w, br, bi);
    }
    if (k < lo) break;
    --j;
    const float s = pow2f(P.piece_delta[j]);
    hr *= s;
    hm *= s;
    k0 = max((long long)P.piece_k0[j], lo);
  }
  rho_lo = P.piece_rho0[j] + (long long)P.piece_beta[j] * (lo - P.piece_k0[j]);
}

// bottom-up over [lo, hi] with multiplier 1/z = u 2^ue: sum b_k 2^rho(k) z^(k-hi) = h 2^rho(hi)
template <bool CC, bool CZ>
__device__ __forceinline__ void window_horner_rev_f32(const DevPoly &P, const cdd &u, int ue, long long lo,
                                                      long long hi, float &hr, float &hm, long long &rho_hi) {
  const float *__restrict__ b = P.bf;
  int j = P.piece_first[lo >> P.log2_piece];
  while (P.piece_k0[j + 1] <= lo) ++j;
  load_bf<CC>(b, lo, hr, hm);
  long long k = lo + 1;
  while (k <= hi) {
    const int sh = ue - P.piece_beta[j];
    const ff2 v = ff_split(scale2(u.rh, sh), CZ ? scale2(u.ih, sh) : 0.0);
    const long long kend = min((long long)P.piece_k0[j + 1] - 1, hi);
#pragma unroll 4
    for (; k <= kend; ++k) {
      float br, bi;
      load_bf<CC>(b, k, br, bi);
      ff_step<CC, CZ>(hr, hm, v, br, bi);
    }
    if (k > hi) break;
    // k is the first index of piece j + 1: rescale, one step with v_j, then piece j + 1
    const float s = pow2f(-P.piece_delta[j]);
    hr *= s;
    hm *= s;
    float br, bi;
    load_bf<CC>(b, k, br, bi);
    ff_step<CC, CZ>(hr, hm, v, br, bi);
    ++k;
    ++j;
  }
  rho_hi = P.piece_rho0[j] + (long long)P.piece_beta[j] * (hi - P.piece_k0[j]);
}

// FP32 counterpart of range_sum with xd values: u = 1/m in plain FP64
// (u.rh, u.ih), which the float-float multiplier of the bottom-up part is
// split from anyway.
template <bool CC, bool CZ>
__device__ __forceinline__ xd range_sum_f32x(const DevPoly &P, double zr, double zi, double mr, double mi, int f,
                                             const cdd &u, long long lo, long long hi, long long kl,
                                             long long &base) {
  xd X = {0.0, 0.0, 0};
  const long long top_lo = max(kl, lo);
  const long long low_hi = min(top_lo - 1, hi);
  const bool has_up = top_lo <= hi, has_low = lo <= low_hi;
  if (has_up) {
    float hr, hm;
    long long rho;
    window_horner_f32<CC, CZ>(P, zr, zi, top_lo, hi, hr, hm, rho);
    X = xd_norm((double)hr, (double)hm, rho);
    base = top_lo;
  }
  if (has_low) {
    float hr, hm;
    long long rho;
    window_horner_rev_f32<CC, CZ>(P, u, -f, lo, low_hi, hr, hm, rho);
    if (has_up && (X.r != 0.0 || X.i != 0.0)) X = xd_mul_d(X, mr, mi, f);
    X = xd_add(X, xd_norm((double)hr, (double)hm, rho));
    base = low_hi;
  }
  return X;
}

// 1/m for a unit-size complex m in plain FP64, as a cdd with zero low parts
__device__ __forceinline__ cdd recip_d(double mr, double mi) {
  const double inv = 1.0 / fma(mr, mr, mi * mi);
  return {mr * inv, 0.0, -mi * inv, 0.0};
}

// Integer-pipe Horner continued from g (scaled at index k + 1, which lies in
// piece j) down to lo: g <- g 2^(rho(k+1) - rho(k)) w' + i^t b_k with the
// packed coefficients, t advancing by -q (mod 4) per step (w = i^q w').
// t on entry is the rotation of the first step's coefficient.  Returns the
// piece holding lo.
template <bool CC, bool CZ, bool SPLIT>
__device__ __forceinline__ int int_horner(const DevPoly &P, isum &h, const iw &w, long long k, int j, long long lo,
                                          int t) {
  const int dq = (4 - w.q) & 3;
  while (k >= lo) {
    if (k < P.piece_k0[j]) {
      --j;  // k == piece_k0[j + 1] - 1: enter piece j
      h.G += P.piece_delta[j];
    }
    const int we64 = w.E + P.piece_beta[j] + 64;
    const long long k0 = max((long long)P.piece_k0[j], lo);
    if (CC) {
      const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(P.bq);
      for (; k - (kIsumMaxSteps - 1) >= k0; k -= kIsumMaxSteps) {
#pragma unroll
        for (int u = 0; u < kIsumMaxSteps; ++u) {
          const ulonglong2 c = __ldg(&b2[k - u]);
          isum_step<CC, CZ, SPLIT>(h, w, we64, c.x, c.y, t);
          t = (t + dq) & 3;
        }
        isum_normalise(h);
      }
      for (; k >= k0; --k) {
        const ulonglong2 c = __ldg(&b2[k]);
        isum_step<CC, CZ, SPLIT>(h, w, we64, c.x, c.y, t);
        t = (t + dq) & 3;
      }
    } else {
      const unsigned long long *b1 = reinterpret_cast<const unsigned long long *>(P.bq);
      for (; k - (kIsumMaxSteps - 1) >= k0; k -= kIsumMaxSteps) {
#pragma unroll
        for (int u = 0; u < kIsumMaxSteps; ++u) {
          isum_step<CC, CZ, SPLIT>(h, w, we64, __ldg(&b1[k - u]), 0ull, t);
          t = (t + dq) & 3;
        }
        isum_normalise(h);
      }
      for (; k >= k0; --k) {
        isum_step<CC, CZ, SPLIT>(h, w, we64, __ldg(&b1[k]), 0ull, t);
        t = (t + dq) & 3;
      }
    }
    isum_normalise(h);  // at most kIsumMaxSteps - 1 steps since the last one
  }
  return j;
}

// Continue the Horner sum g = h (the value at index top, scaled by
// 2^rho(top)) on the integer pipe down to lo; returns sum_{k=lo}^{..}
// a_k z^(k - lo) as extended double-double.
template <bool CC, bool CZ>
__device__ __forceinline__ xint int_tail_x(const DevPoly &P, isum h, double zr, double zi, long long top,
                                           long long lo) {
  int j = P.piece_first[top >> P.log2_piece];
  while (P.piece_k0[j + 1] <= top) ++j;
  const iw w = iw_from(zr, CZ ? zi : 0.0);
  const int t0 = (4 - w.q) & 3;
  if (CZ && w.split)
    j = int_horner<CC, CZ, true>(P, h, w, top - 1, j, lo, t0);
  else
    j = int_horner<CC, CZ, false>(P, h, w, top - 1, j, lo, t0);
  isum_rotate(h, (int)((w.q * ((top - lo) & 3)) & 3));  // h = i^(q (top - lo)) g
  xint X = xint_from_isum(h);
  if (X.x || X.y) X.e += P.piece_rho0[j] + (long long)P.piece_beta[j] * (lo - P.piece_k0[j]);
  return X;
}
template <bool CC, bool CZ>
__device__ __forceinline__ xdd int_tail(const DevPoly &P, isum h, double zr, double zi, long long top, long long lo) {
  return xdd_from_xint(int_tail_x<CC, CZ>(P, h, zr, zi, top, lo));
}

// sum_{k=lo}^{hi} a_k z^(k - lo) in extended double-double by Horner taken
// top-down on the integer pipe (FPE_ACCURATE): every step rounds at 2^-104
// or less of the partial sum, so the order that makes FP64 accurate (toward
// the peak term) is not needed and no FP64 instruction is spent.
template <bool CC, bool CZ>
__device__ __forceinline__ xint window_sum_int_x(const DevPoly &P, double zr, double zi, long long lo,
                                                 long long hi) {
  isum h;
  if (CC) {
    const double2 c = reinterpret_cast<const double2 *>(P.b)[hi];
    h = isum_from(c.x, c.y);
  } else {
    h = isum_from(P.b[hi], 0.0);
  }
  return int_tail_x<CC, CZ>(P, h, zr, zi, hi, lo);
}
template <bool CC, bool CZ>
__device__ __forceinline__ xdd window_sum_int(const DevPoly &P, double zr, double zi, long long lo, long long hi) {
  return xdd_from_xint(window_sum_int_x<CC, CZ>(P, zr, zi, lo, hi));
}

// Sparse windows: when at most a quarter of [lo, hi] lies in G_p, Horner's
// scheme runs over the good indices alone, X <- X z^(k' - k) + a_k, in 128-bit
// fixed point on the integer pipe (every product and sum rounds at 2^-120 or
// less of its operands, so the result is within L 2^-119 S of the window
// sum; no certificate is needed).  The powers come by binary powering; a_k =
// b_k 2^rho(k) exactly.  Returns sum_{good k in [lo, hi]} a_k z^(k - lo).
__device__ __forceinline__ bool sparse_window(const DevPoly &P, long long lo, long long hi) {
  if (P.sparse_mode) return P.sparse_mode == 2;
  const long long g = P.gcount[hi + 1] - P.gcount[lo];
  return 4 * g < hi - lo + 1;
}
template <bool CC>
__device__ __forceinline__ xint window_sum_sparse(const DevPoly &P, double zr, double zi, int f, long long lo,
                                                  long long hi) {
  const int g0 = P.gcount[lo], g1 = P.gcount[hi + 1];
  xint X = xint_norm(0, 0, 0, 0, 0);
  if (g0 >= g1) return X;
  auto coef = [&](long long k, int &j) {  // a_k as an xint; j: a piece at or above k's, moved down to it
    while (P.piece_k0[j] > k) --j;
    const long long rho = P.piece_rho0[j] + (long long)P.piece_beta[j] * (k - P.piece_k0[j]);
    double br, bi = 0.0;
    if (CC) {
      const double2 c = __ldg(reinterpret_cast<const double2 *>(P.b) + k);
      br = c.x;
      bi = c.y;
    } else {
      br = __ldg(P.b + k);
    }
    return xint_from_dd2(br, 0.0, bi, 0.0, rho);
  };
  long long k = __ldg(P.good_idx + g1 - 1);
  int j = P.piece_first[k >> P.log2_piece];
  while (P.piece_k0[j + 1] <= k) ++j;
  X = coef(k, j);
  for (int g = g1 - 2; g >= g0; --g) {
    const long long k2 = __ldg(P.good_idx + g);
    X = xint_add(xint_mul(X, xint_pow_z(zr, zi, k - k2, f)), coef(k2, j));
    k = k2;
  }
  if (k > lo && (X.x || X.y)) X = xint_mul(X, xint_pow_z(zr, zi, k - lo, f));
  return X;
}

// Appends bucketed position q to the list of windows to sum again exactly
// (one atomic per warp for the lanes that call it together).
__device__ __forceinline__ void list_resum(uint32_t *cnt, uint32_t *list, int q) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(&cnt[kCntResum], (unsigned)__popc(m));
  base = __shfl_sync(m, base, leader);
  list[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)q;
}

// a b for xints of which only the parts the flags allow are nonzero: VC, a
// complex; MC, b complex.  Real operands take one 128-bit product instead of
// four, with the result xint_mul would give.
template <bool VC, bool MC>
__device__ __forceinline__ xint xint_mul_k(const xint &a, const xint &b) {
  if (MC) return xint_mul(a, b);
  if (!VC) return xint_norm(mulhi128(a.x, b.x), a.sx ^ b.sx, 0, 0, a.e + b.e + 2);
  return xint_norm(mulhi128(a.x, b.x), a.sx ^ b.sx, mulhi128(a.y, b.x), a.sy ^ b.sx, a.e + b.e + 2);
}

// z^n (n >= 0) by binary powering on the integer pipe; CZ false: z real
template <bool CZ>
__device__ __forceinline__ xint xint_pow_z_k(double zr, double zi, long long n, int f) {
  if (CZ || n <= 0) return xint_pow_z(zr, zi, n, f);
  const double mr = scale2(zr, -f);
  const xint z = xint_norm(u128_from_unit(mr), mr < 0.0, 0, 0, -1);
  xint r = z;
  for (int b = 62 - __clzll(n); b >= 0; --b) {
    r = xint_mul_k<false, false>(r, r);
    if ((n >> b) & 1) r = xint_mul_k<false, false>(r, z);
  }
  r.e += (long long)f * n;
  return r;
}

// One point of a short window (L <= the long-window threshold), or a special point: its
// window's sum, then the power z^(base + v).  A default-mode
// FP64 sum that fails its certificate is listed (resum, at bucketed position q) for
// k_resum and its point left to it.
template <bool CC, bool CZ, bool ACC, bool F32, bool BATCH>
__device__ __forceinline__ void sum_point(const DevPoly &P0, const DevPoly *__restrict__ table,
                                          const PointRec &r, int q, uint32_t *cnt, uint32_t *resum,
                                          fpe_xc64 *__restrict__ out, int32_t *nterms, int32_t *bits_lost) {
  const DevPoly &P = BATCH ? table[r.pid] : P0;
  fpe_xc64 o;
  if (r.flags) {
    o = special_value(P, r.flags);
  } else {
    long long base = r.lo;
    if (F32) {  // xd values: the mode's tolerance does not need double-double
      const int f = frexp_exp(fmax(fabs(r.zr), fabs(r.zi)));
      const double mr = scale2(r.zr, -f), mi = scale2(r.zi, -f);
      cdd u = {0.0, 0.0, 0.0, 0.0};
      if (r.lo < r.kl) u = recip_d(mr, mi);
      const xd X = range_sum_f32x<CC, CZ>(P, r.zr, r.zi, mr, mi, f, u, r.lo, r.hi, r.kl, base);
      const xd v = xd_mul(X, xd_pow_int(r.zr, r.zi, base + P.v));
      o.re = v.r;
      o.im = v.i;
      o.e = v.e;
    } else {
      if (sparse_window(P, r.lo, r.hi)) {
        const int f = frexp_exp(fmax(fabs(r.zr), fabs(r.zi)));
        const xint X = window_sum_sparse<CC>(P, r.zr, CZ ? r.zi : 0.0, f, r.lo, r.hi);
        o = xc64_from_xint(xint_mul(X, xint_pow_z(r.zr, CZ ? r.zi : 0.0, r.lo + P.v, f)));
      } else if (ACC || (!CC && !CZ)) {
        // FPE_ACCURATE, and real points with real coefficients in every mode:
        // the window exactly on the integer pipe (for real arithmetic this
        // costs less on this GPU than the FP64 pass with its certificate and
        // the re-sums of the windows it rejects), z^(l + v) likewise
        const int f = frexp_exp(fmax(fabs(r.zr), fabs(r.zi)));
        const xint X = window_sum_int_x<CC, CZ>(P, r.zr, r.zi, r.lo, r.hi);
        o = xc64_from_xint(xint_mul_k<CC || CZ, CZ>(X, xint_pow_z_k<CZ>(r.zr, r.zi, r.lo + P.v, f)));
      } else {  // bookkeeping in fixed point (integer pipe): 1/z, its powers, the final product
        const int f = frexp_exp(fmax(fabs(r.zr), fabs(r.zi)));
        const double mr = scale2(r.zr, -f), mi = scale2(r.zi, -f);
        xint u = xint_norm(0, 0, 0, 0, 0);
        if (r.lo < r.kl) u = recip_xint(mr, mi);
        bool ok;
        const xint X = range_sum<CC, CZ>(P, r.zr, r.zi, mr, mi, f, u, r.lo, r.hi, r.kl, base, ok);
        if (!ok) {  // not certified: k_resum sums the window exactly
          list_resum(cnt, resum, q);
          return;
        }
        o = xc64_from_xint(xint_mul(X, xint_pow_z(r.zr, r.zi, base + P.v, f)));
      }
    }
  }
  out[r.orig] = o;
  write_diag(P, r, o, nterms, bits_lost);
}

__device__ __forceinline__ xdd shfl_down_xdd(xdd x, int s) {
  xdd y;
  y.rh = __shfl_down_sync(0xffffffffu, x.rh, s);
  y.rl = __shfl_down_sync(0xffffffffu, x.rl, s);
  y.ih = __shfl_down_sync(0xffffffffu, x.ih, s);
  y.il = __shfl_down_sync(0xffffffffu, x.il, s);
  y.e = __shfl_down_sync(0xffffffffu, x.e, s);
  return y;
}
__device__ __forceinline__ xdd shfl_xor_xdd(xdd x, int s) {
  xdd y;
  y.rh = __shfl_xor_sync(0xffffffffu, x.rh, s);
  y.rl = __shfl_xor_sync(0xffffffffu, x.rl, s);
  y.ih = __shfl_xor_sync(0xffffffffu, x.ih, s);
  y.il = __shfl_xor_sync(0xffffffffu, x.il, s);
  y.e = __shfl_xor_sync(0xffffffffu, x.e, s);
  return y;
}
__device__ __forceinline__ xdd shfl_up_xdd(xdd x, int s) {
  xdd y;
  y.rh = __shfl_up_sync(0xffffffffu, x.rh, s);
  y.rl = __shfl_up_sync(0xffffffffu, x.rl, s);
  y.ih = __shfl_up_sync(0xffffffffu, x.ih, s);
  y.il = __shfl_up_sync(0xffffffffu, x.il, s);
  y.e = __shfl_up_sync(0xffffffffu, x.e, s);
  return y;
}

// warp shuffles of an xint: mode 0 up, 1 down, 2 xor
__device__ __forceinline__ xint shfl_xint(const xint &v, int sft, int mode) {
  auto sh64 = [sft, mode](unsigned long long x) -> unsigned long long {
    return mode == 0 ? __shfl_up_sync(0xffffffffu, x, sft)
                     : (mode == 1 ? __shfl_down_sync(0xffffffffu, x, sft) : __shfl_xor_sync(0xffffffffu, x, sft));
  };
  auto sh32 = [sft, mode](int x) -> int {
    return mode == 0 ? __shfl_up_sync(0xffffffffu, x, sft)
                     : (mode == 1 ? __shfl_down_sync(0xffffffffu, x, sft) : __shfl_xor_sync(0xffffffffu, x, sft));
  };
  xint r;
  r.x = ((u128)sh64((unsigned long long)(v.x >> 64)) << 64) | sh64((unsigned long long)v.x);
  r.y = ((u128)sh64((unsigned long long)(v.y >> 64)) << 64) | sh64((unsigned long long)v.y);
  r.sx = sh32(v.sx);
  r.sy = sh32(v.sy);
  r.e = (long long)sh64((unsigned long long)v.e);
  return r;
}

// Long windows: warp groups.  A window of length L gets ng = ceil(L / (32 lane_chunk))
// groups of S = 32 C terms with C = ceil(L / (32 ng)); lane i of group g owns
// the chunk [c_i, c_i + C - 1], c_i = l + g S + i C, and a slot value s_i with
//   sum over the window = z^l sum_g (z^S)^g sum_i (z^C)^i s_i.
// FP64 precision: s_i = sum a_k z^(k - c_i), exactly on the integer pipe, and
// the group's value sum_i (z^C)^i s_i by a tree over the lanes (lanes_tree).
// FP32 mode: FP32 passes toward the peak, so a chunk below the peak hands its
// sum z^(c_{i+1} - 1) R to slot i+1 as R / z (the group's carry out of lane
// 31 goes to the next group), the chunk holding the peak sums both parts, and
// each lane scales its slot by its own power before a butterfly adds them.
// The warp that finishes a window's last group combines the groups and
// applies z^(l + v).
__device__ __forceinline__ int group_slot(int i, int g, int gbase, int cap) {
  return g == 0 ? i : cap + gbase + g - 1;
}

// One thread per bucketed point with a short window (static blocks).
template <bool CC, bool CZ, bool ACC, bool F32, bool BATCH>
__global__ void __launch_bounds__(128, kSumBlocksPerSm) k_sum_short(DevPoly P0, const DevPoly *__restrict__ table,
                                                                    int n, const PointRec *__restrict__ rec,
                                                                    fpe_xc64 *__restrict__ out, int32_t *nterms,
                                                                    int32_t *bits_lost, long long long_window,
                                                                    uint32_t *cnt, uint32_t *resum) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const PointRec r = rec[q];
  if (r.flags & kPointTC) return;
  if (r.flags || r.hi - r.lo + 1 <= long_window)
    sum_point<CC, CZ, ACC, F32, BATCH>(P0, table, r, q, cnt, resum, out, nterms, bits_lost);
}

// sum_i (z^C)^i v_i over the 32 lanes' values, into lane 0, by a tree: at
// level s = 1, 2, 4, 8, 16 every lane adds the value of lane + s times
// Z^s (Z = z^C, squared between levels).  Lane i with i a multiple of 2s then
// holds sum_{j < 2s} Z^j v_(i+j); the other lanes' values are never read by
// lane 0.  Every lane runs the same steps: no lane waits on another's branch.
template <bool VC, bool CZ>
__device__ __forceinline__ xint lanes_tree(xint v, double zr, double zi, long long C, int f) {
  xint Z = xint_pow_z_k<CZ>(zr, zi, C, f);
#pragma unroll 1
  for (int s = 1; s < 32; s <<= 1) {
    const xint o = shfl_xint(v, s, 1);
    v = xint_add(v, xint_mul_k<VC || CZ, CZ>(o, Z));
    if (s < 16) Z = CZ ? xint_sqr(Z) : xint_mul_k<false, false>(Z, Z);
  }
  return v;
}

// Group g of a long window (ng groups): lane i sums its chunk, the 32 slots
// are combined; lane 0 returns the group's value sv and carry gout.
template <bool CC, bool CZ, bool ACC, bool F32>
__device__ __forceinline__ void sum_group(const DevPoly &P, const PointRec &r, int ng, int g, int lane, uint32_t *cnt,
                                          xdd &sv_out, xdd &gout_out) {
  const long long L = r.hi - r.lo + 1;
  const long long C = (L + 32LL * ng - 1) / (32LL * ng);
  const long long clo = r.lo + (long long)g * 32 * C + lane * C;
  const long long chi = min(clo + C - 1, r.hi);
  if constexpr (F32) {  // the same steps in xd values
    xd v = {0.0, 0.0, 0}, cy = {0.0, 0.0, 0};
    if (clo <= chi) {
      const int f = frexp_exp(fmax(fabs(r.zr), fabs(r.zi)));
      const double mr = scale2(r.zr, -f), mi = scale2(r.zi, -f);
      const cdd u = recip_d(mr, mi);
      long long base;
      const xd X = range_sum_f32x<CC, CZ>(P, r.zr, r.zi, mr, mi, f, u, clo, chi, r.kl, base);
      if (chi < r.kl)
        cy = xd_mul_d(X, u.rh, u.ih, -f);
      else if (base > clo)
        v = xd_mul(X, xd_pow_int(r.zr, r.zi, base - clo));
      else
        v = X;
    }
    auto shfl = [](xd x, int sft, int mode) {
      xd y;
      if (mode == 0) {
        y.r = __shfl_up_sync(0xffffffffu, x.r, sft);
        y.i = __shfl_up_sync(0xffffffffu, x.i, sft);
        y.e = __shfl_up_sync(0xffffffffu, x.e, sft);
      } else if (mode == 1) {
        y.r = __shfl_down_sync(0xffffffffu, x.r, sft);
        y.i = __shfl_down_sync(0xffffffffu, x.i, sft);
        y.e = __shfl_down_sync(0xffffffffu, x.e, sft);
      } else {
        y.r = __shfl_xor_sync(0xffffffffu, x.r, sft);
        y.i = __shfl_xor_sync(0xffffffffu, x.i, sft);
        y.e = __shfl_xor_sync(0xffffffffu, x.e, sft);
      }
      return y;
    };
    const xd inc = shfl(cy, 1, 0);
    if (lane > 0) v = xd_add(v, inc);
    const xd go = shfl(cy, 31, 1);  // lane 31's carry, read by lane 0
    if (lane > 0 && (v.r != 0.0 || v.i != 0.0)) v = xd_mul(v, xd_pow_int(r.zr, r.zi, lane * C));
    for (int sft = 16; sft >= 1; sft >>= 1) v = xd_add(v, shfl(v, sft, 2));
    sv_out = xdd_from_xd(v);
    gout_out = xdd_from_xd(go);
    return;
  }
  // FP64 precision (either mode): each lane's chunk exactly on the integer
  // pipe, top-down (the order does not matter there).  On this GPU an
  // integer Horner step costs less issue time than an FP64 step with its
  // certificate (one FP64 warp instruction takes as long as about 38 integer
  // ones), and every lane runs the same loop: no split into chunks summed
  // top-down and bottom-up, no re-sum of uncertified chunks.
  const int f = frexp_exp(fmax(fabs(r.zr), fabs(r.zi)));
  xint sv = xint_norm(0, 0, 0, 0, 0);
  if (clo <= chi)
    sv = sparse_window(P, clo, chi) ? window_sum_sparse<CC>(P, r.zr, CZ ? r.zi : 0.0, f, clo, chi)
                                    : window_sum_int_x<CC, CZ>(P, r.zr, r.zi, clo, chi);
  sv = lanes_tree<CC, CZ>(sv, r.zr, r.zi, C, f);
  sv_out = xdd_from_xint(sv);
  gout_out = xdd_zero();
}

// A long window with one group: its value times z^(l + v), written by one thread.
__device__ __forceinline__ void finalize_one(const DevPoly &P, const PointRec &r, const xdd &val,
                                             fpe_xc64 *__restrict__ out, int32_t *nterms, int32_t *bits_lost) {
  const xdd pw = xdd_pow_int(r.zr, r.zi, r.lo + P.v);
  const fpe_xc64 o = xdd_out(xdd_mul(val, pw));
  out[r.orig] = o;
  write_diag(P, r, o, nterms, bits_lost);
}

// The short windows whose FP64 sums failed their certificates (listed by
// sum_point), summed again exactly on the integer pipe (the Horner of
// FPE_ACCURATE).  A window of at most kResumThreadMax terms takes one thread;
// a longer one SEG lanes (8 up to kResumSegMax terms, else a whole warp):
// lane i sums the chunk [l + i C, l + (i + 1) C - 1], C = ceil(L / SEG),
// multiplies it by z^(l + i C + v), and a butterfly over the window's lanes
// adds them, so no lane's chain is long.
constexpr long long kResumThreadMax = 48;
constexpr long long kResumSegMax = 256;
template <bool CC, bool CZ, int SEG>
__device__ __forceinline__ void resum_window(const DevPoly &P, const PointRec &r, bool valid, int sl,
                                             fpe_xc64 *__restrict__ out, int32_t *nterms, int32_t *bits_lost) {
  xdd sv = xdd_zero();
  if (valid) {
    const long long L = r.hi - r.lo + 1, C = (L + SEG - 1) / SEG;
    const long long clo = r.lo + sl * C, chi = min(clo + C - 1, r.hi);
    if (clo <= chi) sv = window_sum_int<CC, CZ>(P, r.zr, r.zi, clo, chi);
    if (sv.rh != 0.0 || sv.ih != 0.0) sv = xdd_mul(sv, xdd_pow_int(r.zr, r.zi, clo + P.v));
  }
  for (int s = SEG / 2; s >= 1; s >>= 1) sv = xdd_add(sv, shfl_xor_xdd(sv, s));
  if (valid && sl == 0) {
    const fpe_xc64 o = xdd_out(sv);
    out[r.orig] = o;
    write_diag(P, r, o, nterms, bits_lost);
  }
}
template <bool CC, bool CZ, bool BATCH>
__global__ void __launch_bounds__(128) k_resum(DevPoly P0, const DevPoly *__restrict__ table,
                                               const PointRec *__restrict__ rec, const uint32_t *cnt,
                                               const uint32_t *__restrict__ list, fpe_xc64 *__restrict__ out,
                                               int32_t *nterms, int32_t *bits_lost) {
  const uint32_t m = *(volatile const uint32_t *)&cnt[kCntResum];
  const int lane = threadIdx.x & 31;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  for (uint32_t i = tid; i < m; i += nthr) {  // the shortest, a thread each
    const PointRec r = rec[list[i]];
    if (r.hi - r.lo + 1 > kResumThreadMax) continue;
    const DevPoly &P = BATCH ? table[r.pid] : P0;
    const xdd Y = window_sum_int<CC, CZ>(P, r.zr, r.zi, r.lo, r.hi);
    const fpe_xc64 o = xdd_out(xdd_mul(Y, xdd_pow_int(r.zr, r.zi, r.lo + P.v)));
    out[r.orig] = o;
    write_diag(P, r, o, nterms, bits_lost);
  }
  const uint32_t wid = tid >> 5, nw = nthr >> 5;
  for (uint32_t b = wid * 4; b < m; b += nw * 4) {  // four windows of at most kResumSegMax terms per warp
    const uint32_t i = b + (lane >> 3);
    PointRec r{};
    bool valid = i < m;
    if (valid) {
      r = rec[list[i]];
      const long long L = r.hi - r.lo + 1;
      valid = L > kResumThreadMax && L <= kResumSegMax;
    }
    const DevPoly &P = BATCH ? table[valid ? r.pid : 0] : P0;
    resum_window<CC, CZ, 8>(P, r, valid, lane & 7, out, nterms, bits_lost);
  }
  for (uint32_t i = wid; i < m; i += nw) {  // the longer ones, a warp each
    const PointRec r = rec[list[i]];
    if (r.hi - r.lo + 1 <= kResumSegMax) continue;  // warp-uniform
    const DevPoly &P = BATCH ? table[r.pid] : P0;
    resum_window<CC, CZ, 32>(P, r, true, lane, out, nterms, bits_lost);
  }
}

// Warp groups of the long windows, one evaluation of one polynomial:
// persistent warps take group items from a counter and store each group's
// value and carry; k_finalize_long combines them.
template <bool CC, bool CZ, bool ACC, bool F32>
__global__ void __launch_bounds__(128, kSumBlocksPerSm) k_sum_groups(
    DevPoly P, const PointRec *__restrict__ rec, const int32_t *__restrict__ long_list,
    const int32_t *__restrict__ long_ngroups, const int32_t *__restrict__ long_gbase,
    const int32_t *__restrict__ extra_owner, const int32_t *__restrict__ extra_group, uint32_t *cnt, int cap,
    int extra_cap, xdd *__restrict__ gval, xdd *__restrict__ gcarry) {
  const int lane = threadIdx.x & 31;
  const uint32_t nlong = *(volatile uint32_t *)&cnt[kCntLong];
  // every extra slot below min(reserved, extra_cap) is written by the scatter: an owner, or -1
  const uint32_t nextra = min(*(volatile uint32_t *)&cnt[kCntExtra], (uint32_t)extra_cap);
  while (true) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&cnt[kCntGroupWork], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nlong + nextra) break;
    int i, g;
    if (t < nlong) {
      i = (int)t;
      g = 0;
    } else {
      i = extra_owner[t - nlong];
      if (i < 0) continue;  // slot of a reservation that did not fit
      g = extra_group[t - nlong];
    }
    const PointRec r = rec[long_list[i]];
    xdd sv, gout;
    sum_group<CC, CZ, ACC, F32>(P, r, long_ngroups[i] & 0xffff, g, lane, cnt, sv, gout);
    if (lane == 0) {
      const int slot = group_slot(i, g, long_gbase[i], cap);
      gval[slot] = sv;
      gcarry[slot] = gout;
    }
  }
}

// The warp-parallel combination of a long window's ng > 1 groups (all 32
// lanes call it): lane g holds val_g + carry_{g-1} times W^g = z^(32 C g),
// a butterfly adds the lanes, lane 0 applies z^(l + v) and writes the point.
// Group values written by other SMs are read past L1.
template <bool BATCH>
__device__ __forceinline__ void finalize_warp(const DevPoly &P0, const DevPoly *__restrict__ table,
                                              const PointRec &r, int i, int ng, int gb, int cap,
                                              const xdd *gval, const xdd *gcarry, int lane,
                                              fpe_xc64 *__restrict__ out, int32_t *nterms, int32_t *bits_lost) {
  const DevPoly &P = BATCH ? table[r.pid] : P0;
  auto ld = [](const xdd *p) {
    xdd x;
    x.rh = __ldcg(&p->rh);
    x.rl = __ldcg(&p->rl);
    x.ih = __ldcg(&p->ih);
    x.il = __ldcg(&p->il);
    x.e = __ldcg(&p->e);
    return x;
  };
  const long long L = r.hi - r.lo + 1;
  const long long C = (L + 32LL * ng - 1) / (32LL * ng);
  auto slot_sum = [&](int g) {  // val_g + carry_{g-1}
    xdd v = ld(&gval[group_slot(i, g, gb, cap)]);
    if (g > 0) v = xdd_add(v, ld(&gcarry[group_slot(i, g - 1, gb, cap)]));
    return v;
  };
  xdd t = xdd_zero();
  if (ng <= 32) {
    if (lane < ng) t = slot_sum(lane);
  } else {  // the lane's groups lane + 32 m, by Horner in W^32 from the top m
    const xdd W32 = xdd_pow_int(r.zr, r.zi, 32 * 32 * C);
    for (int g = lane + 32 * ((ng - 1 - lane) / 32); g >= lane; g -= 32) t = xdd_add(xdd_mul(t, W32), slot_sum(g));
  }
  // lane 0: z^(l + v); lane g > 0: W^g
  const xdd pw = xdd_pow_int(r.zr, r.zi, lane == 0 ? r.lo + P.v : 32 * C * lane);
  if (lane > 0 && (t.rh != 0.0 || t.ih != 0.0)) t = xdd_mul(t, pw);
  for (int sft = 16; sft >= 1; sft >>= 1) t = xdd_add(t, shfl_xor_xdd(t, sft));
  if (lane == 0) {
    const fpe_xc64 o = xdd_out(xdd_mul(t, pw));
    out[r.orig] = o;
    write_diag(P, r, o, nterms, bits_lost);
  }
}

// Finish the long windows.  A window with one group takes one thread: its
// power z^(l + v) and one product.  A window with ng > 1 groups takes a warp:
// lane g holds group g's value plus the carry of group g - 1 and multiplies
// it by its own power W^g = z^(32 C g) (integer pipe), a butterfly adds the
// lanes, and lane 0, which meanwhile computed z^(l + v), writes the point.
// (On this GPU a dependent FP64 instruction costs a warp tens of cycles, so
// a one-thread Horner over 32 groups in double-double was the kernel's
// whole duration.)  For ng > 32 lane g first sums its groups g + 32 m by
// Horner in W^32.
__global__ void __launch_bounds__(128) k_finalize_long(DevPoly P, const PointRec *__restrict__ rec,
                                                       const int32_t *__restrict__ long_list,
                                                       const int32_t *__restrict__ long_ngroups,
                                                       const int32_t *__restrict__ long_gbase, const uint32_t *cnt,
                                                       int cap, const xdd *__restrict__ gval,
                                                       const xdd *__restrict__ gcarry, fpe_xc64 *__restrict__ out,
                                                       int32_t *nterms, int32_t *bits_lost) {
  const uint32_t nlong = *(volatile const uint32_t *)&cnt[kCntLong];
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  for (uint32_t i = tid; i < nlong; i += nthr) {
    if ((long_ngroups[i] & 0xffff) != 1) continue;
    const PointRec r = rec[long_list[i]];
    finalize_one(P, r, gval[group_slot((int)i, 0, long_gbase[i], cap)], out, nterms, bits_lost);
  }
  const int lane = threadIdx.x & 31;
  const uint32_t wid = tid >> 5, nwarps = nthr >> 5;
  for (uint32_t i = wid; i < nlong; i += nwarps) {
    const int ng = long_ngroups[i] & 0xffff;
    if (ng == 1) continue;  // warp-uniform
    finalize_warp<false>(P, nullptr, rec[long_list[i]], (int)i, ng, long_gbase[i], cap, gval, gcarry, lane, out,
                         nterms, bits_lost);
  }
}

// All window sums of one batched evaluation in one persistent launch (the
// single-polynomial path uses k_sum_short, k_sum_groups, k_finalize_long,
// which measured faster there).  Each warp
// takes work items from a counter:
//   first the warp groups of the long windows (the largest items), a group
//   being 32 lane chunks of one window (see above);
//   then 32 consecutive bucketed points each, one per lane, whose short
//   windows (or special values) fill the tail.
// A window with one group is finished by the warp that sums it.  Otherwise
// each group stores its value, fences, and counts itself done in the upper
// 16 bits of long_ngroups[i]; the warp that completes the count combines the
// groups (all lanes, finalize_warp) and writes the point.  No warp ever
// waits for another.
template <bool CC, bool CZ, bool ACC, bool F32, bool BATCH>
__global__ void __launch_bounds__(128, kSumBlocksPerSm) k_sums(
    DevPoly P0, const DevPoly *__restrict__ table, int n, const PointRec *__restrict__ rec,
    const int32_t *__restrict__ long_list, int32_t *long_ngroups, const int32_t *__restrict__ long_gbase,
    const int32_t *__restrict__ extra_owner, const int32_t *__restrict__ extra_group, uint32_t *cnt, int cap,
    int extra_cap, xdd *gval, xdd *gcarry, fpe_xc64 *__restrict__ out, int32_t *nterms, int32_t *bits_lost,
    long long long_window, uint32_t *resum) {
  const int lane = threadIdx.x & 31;
  const uint32_t nlong = *(volatile uint32_t *)&cnt[kCntLong];
  // every extra slot below min(reserved, extra_cap) is written by the scatter: an owner, or -1
  const uint32_t nextra = min(*(volatile uint32_t *)&cnt[kCntExtra], (uint32_t)extra_cap);
  const uint32_t ngroup_items = nlong + nextra;
  const uint32_t nitems = ngroup_items + (uint32_t)((n + 31) / 32);
  while (true) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&cnt[kCntGroupWork], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nitems) break;
    if (t >= ngroup_items) {  // 32 short-window points
      const long long q = (long long)(t - ngroup_items) * 32 + lane;
      if (q < n) {
        const PointRec r = rec[q];
        if (r.flags || r.hi - r.lo + 1 <= long_window)
          sum_point<CC, CZ, ACC, F32, BATCH>(P0, table, r, (int)q, cnt, resum, out, nterms, bits_lost);
      }
      continue;
    }
    int i, g;
    if (t < nlong) {
      i = (int)t;
      g = 0;
    } else {
      i = extra_owner[t - nlong];
      if (i < 0) continue;  // slot of a reservation that did not fit
      g = extra_group[t - nlong];
    }
    const int ng = *(volatile int32_t *)&long_ngroups[i] & 0xffff;
    const PointRec r = rec[long_list[i]];
    const DevPoly &P = BATCH ? table[r.pid] : P0;
    xdd sv, gout;
    sum_group<CC, CZ, ACC, F32>(P, r, ng, g, lane, cnt, sv, gout);
    if (ng == 1) {  // the whole window: finish it here
      if (lane == 0) finalize_one(P, r, sv, out, nterms, bits_lost);
    } else {
      const int gb = long_gbase[i];
      int last = 0;
      if (lane == 0) {
        const int slot = group_slot(i, g, gb, cap);
        gval[slot] = sv;
        gcarry[slot] = gout;
        __threadfence();  // the group's value is visible before it is counted
        const int done = (int)(atomicAdd(reinterpret_cast<unsigned int *>(&long_ngroups[i]), 1u << 16) >> 16);
        last = done == ng - 1;
      }
      if (__shfl_sync(0xffffffffu, last, 0)) {
        __threadfence();
        finalize_warp<BATCH>(P0, table, r, i, ng, gb, cap, gval, gcarry, lane, out, nterms, bits_lost);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <bool CC, bool CZ, bool ACC, bool F32>
static void launch_sums4(fpe_poly_s *P, int n, fpe_xc64 *out, int32_t *nterms, int32_t *bits_lost,
                         cudaStream_t st, int short_threads) {
  Workspace &w = P->ws;
  const int cap = (int)w.cap, xcap = (int)w.extra_cap;
  uint32_t *cnt = w.bins + 2 * w.nbins;
  {
    ProfScope ps("k_sum_short", st);
    k_sum_short<CC, CZ, ACC, F32, false><<<(n + short_threads - 1) / short_threads, short_threads, 0, st>>>(
        P->dev, nullptr, n, w.rec, out, nterms, bits_lost, P->tune.long_window, cnt, w.key);
  }
  if (!ACC && !F32) {
    ProfScope ps("k_resum", st);
    k_resum<CC, CZ, false><<<num_sms() * 6, 128, 0, st>>>(P->dev, nullptr, w.rec, cnt, w.key, out, nterms, bits_lost);
  }
  {
    ProfScope ps("k_sum_groups", st);
    k_sum_groups<CC, CZ, ACC, F32><<<num_sms() * kSumBlocksPerSm, 128, 0, st>>>(
        P->dev, w.rec, w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner, w.extra_group, cnt, cap, xcap,
        (xdd *)w.group_val, (xdd *)w.group_carry);
  }
  {
    ProfScope ps("k_finalize_long", st);
    k_finalize_long<<<num_sms() * 2, 128, 0, st>>>(P->dev, w.rec, w.long_list, w.long_ngroups, w.long_gbase, cnt,
                                                   cap, (const xdd *)w.group_val, (const xdd *)w.group_carry, out,
                                                   nterms, bits_lost);
  }
}

template <bool CC, bool CZ>
static void launch_sums(fpe_poly_s *P, int n, fpe_xc64 *out, int32_t *nterms, int32_t *bits_lost, cudaStream_t st,
                        int short_threads = 128) {
  if (P->dev.fp32)
    launch_sums4<CC, CZ, false, true>(P, n, out, nterms, bits_lost, st, short_threads);
  else if (P->dev.accurate)
    launch_sums4<CC, CZ, true, false>(P, n, out, nterms, bits_lost, st, short_threads);
  else
    launch_sums4<CC, CZ, false, false>(P, n, out, nterms, bits_lost, st, short_threads);
}

// The handle's second stream and its two events, created on first use on the
// current device (the handle's).
static fpe_status ensure_tc_stream(fpe_poly_s *P) {
  if (P->tc_stream && P->tc_fork && P->tc_join) return FPE_OK;
  cudaError_t e = cudaSuccess;
  if (!P->tc_stream) {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetStreamPriorityRange");
    // hi is the numerically smallest value: the greatest priority
    const int prio = FPE_TC_CONCURRENT == 1 ? hi : 0;
    e = cudaStreamCreateWithPriority(&P->tc_stream, cudaStreamNonBlocking, prio);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithPriority");
  }
  if (!P->tc_fork && (e = cudaEventCreateWithFlags(&P->tc_fork, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreateWithFlags");
  if (!P->tc_join && (e = cudaEventCreateWithFlags(&P->tc_join, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreateWithFlags");
  return FPE_OK;
}

// locate, bucket and scatter the points into P->ws.rec (the front of fpe_eval);
// with allow_tc, windows that qualify for the tensor-core sums are bucketed
// apart and marked kPointTC
fpe_status launch_front(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n64, cudaStream_t st,
                        bool allow_tc) {
  fpe_status s = ensure_workspace(P, n64);
  if (s != FPE_OK) return s;
  const int n = (int)n64;
  Workspace &w = P->ws;
  const bool cz = z_im != nullptr;
  const bool tc = allow_tc && tc_enabled(P, cz, n64);
  if (tc && (s = ensure_tc_workspace(P, n64)) != FPE_OK) return s;
  w.nbins = tc ? kNumBins + P->dev.n_tc * kTcBinsPerPiece : kNumBins;  // bins of the pieces that exist
  const long long tcw = tc ? (long long)P->tune.tc_min_window : 0;
  cudaError_t e = cudaMemsetAsync(w.bins, 0, w.nbins * sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int nb = (n + 255) / 256;
  {
    ProfScope ps("k_locate", st);
    if (cz)
      k_locate<true><<<nb, 256, 0, st>>>(P->dev, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, tcw);
    else
      k_locate<false><<<nb, 256, 0, st>>>(P->dev, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, tcw);
  }
  {
    ProfScope ps("k_scan_bins", st, 2);  // k_scan_tiles, k_scan_bins
    launch_scan_bins(w.bins, w.nbins, st);
  }
  {
    ProfScope ps("k_scatter", st);
    if (cz)
      k_scatter<true><<<nb, 256, 0, st>>>(P->dev, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, w.rec,
                                          w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner,
                                          w.extra_group, (int)w.extra_cap, P->d_status, P->tune.long_window,
                                          P->tune.group_span(), w.nbins);
    else
      k_scatter<false><<<nb, 256, 0, st>>>(P->dev, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, w.rec,
                                           w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner,
                                           w.extra_group, (int)w.extra_cap, P->d_status, P->tune.long_window,
                                           P->tune.group_span(), w.nbins);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  if (tc) return launch_tc_groups(P, n, st);
  return FPE_OK;
}

fpe_status launch_eval(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n64, fpe_xc64 *out,
                       int32_t *nterms, int32_t *bits_lost, cudaStream_t st) {
  if (n64 == 0) return FPE_OK;
  fpe_status s = launch_front(P, z_re, z_im, n64, st, true);
  if (s != FPE_OK) return s;
  const int n = (int)n64;
  const bool cz = z_im != nullptr;
  const bool cc = P->complex_coef;
  const bool tc = P->ws.nbins > kNumBins;
  // With the tensor-core path the two kinds of window sums share nothing but
  // the bucketed records (read only) and disjoint counters, and write
  // disjoint outputs, so by default they run at once: the tensor-core branch
  // (plan, slices, MMAs, finalize) on the handle's second stream, forked from
  // st after the front and joined back into st.  Each SM then keeps its FP64
  // pipe busy with k_sum_short beside the tensor and integer pipes' work.
  cudaStream_t sf = st;  // the FP64 sums' stream
  cudaStream_t stc = st;  // the tensor-core branch's stream
  int short_threads = 128;
  if (tc && FPE_TC_CONCURRENT != 0) {
    if ((s = ensure_tc_stream(P)) != FPE_OK) return s;
    cudaError_t e = cudaEventRecord(P->tc_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->tc_stream, P->tc_fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core stream fork");
    stc = P->tc_stream;
    short_threads = kShortThreadsTc;
  }
  fpe_status stc_status = FPE_OK;
  if (tc) {
    stc_status = launch_tc_plan(P, n, stc);
    if (stc_status == FPE_OK) stc_status = launch_tc_sums(P, n, out, nterms, bits_lost, stc);
  }
  if (cc && cz)
    launch_sums<true, true>(P, n, out, nterms, bits_lost, sf, short_threads);
  else if (cc)
    launch_sums<true, false>(P, n, out, nterms, bits_lost, sf, short_threads);
  else if (cz)
    launch_sums<false, true>(P, n, out, nterms, bits_lost, sf, short_threads);
  else
    launch_sums<false, false>(P, n, out, nterms, bits_lost, sf, short_threads);
  if (stc != st) {  // join, also after a failed launch on the branch
    cudaError_t e = cudaEventRecord(P->tc_join, stc);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P->tc_join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core stream join");
  }
  if (stc_status != FPE_OK) return stc_status;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  P->last_n = n64;
  return FPE_OK;
}

}  // namespace fpe

namespace fpe {

// ---------------------------------------------------------------------------
// Batched evaluation: many polynomials, each at its own points, in one fixed
// sequence of launches (§8.1: points are independent).  The polynomials'
// descriptors live in a device table; every point carries its polynomial's
// index.  Bucketing is a segmented counting sort: kBatchBins lambda bins per
// polynomial, scanned per polynomial, so points stay inside their
// polynomial's segment and a warp's lanes share one coefficient array.
// ---------------------------------------------------------------------------
template <bool CZ>
__global__ void k_locate_batch(const DevPoly *__restrict__ table, const int32_t *__restrict__ pid, int n,
                               const double *__restrict__ zre, const double *__restrict__ zim,
                               long long *__restrict__ lo_out, long long *__restrict__ hi_out,
                               long long *__restrict__ kl_out, double *__restrict__ N_out,
                               uint32_t *__restrict__ key, uint32_t *__restrict__ hist) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int i = pid[p];
  const DevPoly &P = table[i];
  double zr = zre[p], zi = CZ ? zim[p] : 0.0;
  Window w = locate_point<CZ>(P, zr, zi);
  lo_out[p] = w.lo + (w.flags ? 0 : P.v);
  hi_out[p] = w.hi + (w.flags ? 0 : P.v);
  kl_out[p] = w.kl;
  N_out[p] = w.flags ? 0.0 : w.N + w.lam * (double)P.v;
  const uint32_t k = (uint32_t)i * kBatchBins + (bucket_of(w.lam, w.flags) * kBatchBins) / kNumBins;
  key[p] = k;
  atomicAdd(&hist[k], 1u);
}

// per polynomial: exclusive scan of its bins, starting at its first point; resets the counters
__global__ void k_scan_batch(const int64_t *__restrict__ offsets, int npoly, const uint32_t *__restrict__ hist,
                             uint32_t *__restrict__ cursor, uint32_t *__restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNumCounters) cnt[i] = 0;
  if (i >= npoly) return;
  uint32_t run = (uint32_t)offsets[i];
  for (int b = 0; b < kBatchBins; ++b) {
    cursor[i * kBatchBins + b] = run;
    run += hist[i * kBatchBins + b];
  }
}

template <bool CZ>
__global__ void k_scatter_batch(const DevPoly *__restrict__ table, const int32_t *__restrict__ pid, int n,
                                const double *__restrict__ zre, const double *__restrict__ zim,
                                const long long *__restrict__ lo, const long long *__restrict__ hi,
                                const long long *__restrict__ kl, const double *__restrict__ N,
                                const uint32_t *__restrict__ key, uint32_t *cursor, uint32_t *cnt,
                                PointRec *__restrict__ rec, int32_t *__restrict__ long_list,
                                int32_t *__restrict__ long_ngroups, int32_t *__restrict__ long_gbase,
                                int32_t *__restrict__ extra_owner, int32_t *__restrict__ extra_group, int extra_cap,
                                int32_t *status, long long long_window, long long span) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int i = pid[p];
  const long long v = table[i].v;
  uint32_t pos = atomicAdd(&cursor[key[p]], 1u);
  PointRec r;
  r.zr = zre[p];
  r.zi = CZ ? zim[p] : 0.0;
  r.flags = 0;
  if (!isfinite(r.zr) || !isfinite(r.zi)) {
    r.flags = kPointNonFinite;
    atomicOr(status, kStatusNonFinite);
  } else if (r.zr == 0.0 && r.zi == 0.0) {
    r.flags = kPointZero;
  }
  r.lo = r.flags ? 1 : lo[p] - v;
  r.hi = r.flags ? 0 : hi[p] - v;
  r.kl = kl[p];
  r.N = N[p];
  r.orig = p;
  r.pid = i;
  r.pad = 0;
  rec[pos] = r;
  if (!r.flags && r.hi - r.lo + 1 > long_window)
    list_long_window(r.hi - r.lo + 1, span, pos, cnt, long_list, long_ngroups, long_gbase, extra_owner, extra_group,
                     extra_cap);
}

template <bool CC, bool CZ, bool ACC, bool F32>
static void launch_batch_sums(fpe_batch_s *B, fpe_xc64 *out, int32_t *nterms, cudaStream_t st) {
  Workspace &w = B->ws;
  ProfScope ps("k_sums", st);
  k_sums<CC, CZ, ACC, F32, true><<<num_sms() * kSumBlocksPerSm, 128, 0, st>>>(
      DevPoly{}, B->d_table, (int)B->ntotal, w.rec, w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner,
      w.extra_group, B->d_cnt, (int)w.cap, (int)w.extra_cap, (xdd *)w.group_val, (xdd *)w.group_carry, out, nterms,
      nullptr, B->tune.long_window, w.key);
  if (!ACC && !F32)
    k_resum<CC, CZ, true><<<num_sms() * 6, 128, 0, st>>>(DevPoly{}, B->d_table, w.rec, B->d_cnt, w.key, out, nterms,
                                                         nullptr);
}

fpe_status launch_batch(fpe_batch_s *B, const double *z_re, const double *z_im, fpe_xc64 *out, int32_t *nterms,
                        cudaStream_t st) {
  if (B->ntotal == 0) return FPE_OK;
  Workspace &w = B->ws;
  const int n = (int)B->ntotal, nb = (n + 255) / 256;
  const bool cz = z_im != nullptr;
  cudaError_t e = cudaMemsetAsync(B->d_hist, 0, B->npoly * kBatchBins * sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  {
    ProfScope ps("k_locate_batch", st);
    if (cz)
      k_locate_batch<true><<<nb, 256, 0, st>>>(B->d_table, B->d_pid, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key,
                                               B->d_hist);
    else
      k_locate_batch<false><<<nb, 256, 0, st>>>(B->d_table, B->d_pid, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key,
                                                B->d_hist);
  }
  {
    ProfScope ps("k_scan_batch", st);
    const int np = (int)B->npoly;
    k_scan_batch<<<(std::max(np, kNumCounters) + 127) / 128, 128, 0, st>>>(B->d_offsets, np, B->d_hist,
                                                                           B->d_cursor, B->d_cnt);
  }
  {
    ProfScope ps("k_scatter_batch", st);
    if (cz)
      k_scatter_batch<true><<<nb, 256, 0, st>>>(B->d_table, B->d_pid, n, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key,
                                                B->d_cursor, B->d_cnt, w.rec, w.long_list, w.long_ngroups,
                                                w.long_gbase, w.extra_owner, w.extra_group, (int)w.extra_cap,
                                                B->d_status, B->tune.long_window, B->tune.group_span());
    else
      k_scatter_batch<false><<<nb, 256, 0, st>>>(B->d_table, B->d_pid, n, z_re, z_im, w.lo, w.hi, w.kl, w.N,
                                                 w.key, B->d_cursor, B->d_cnt, w.rec, w.long_list, w.long_ngroups,
                                                 w.long_gbase, w.extra_owner, w.extra_group, (int)w.extra_cap,
                                                 B->d_status, B->tune.long_window, B->tune.group_span());
  }
  const bool cc = B->complex_coef;
#define FPE_BATCH_SUMS(CCv, CZv)                                         \
  do {                                                                   \
    if (B->fp32)                                                         \
      launch_batch_sums<CCv, CZv, false, true>(B, out, nterms, st);      \
    else if (B->accurate)                                                \
      launch_batch_sums<CCv, CZv, true, false>(B, out, nterms, st);      \
    else                                                                 \
      launch_batch_sums<CCv, CZv, false, false>(B, out, nterms, st);     \
  } while (0)
  if (cc && cz) FPE_BATCH_SUMS(true, true);
  else if (cc) FPE_BATCH_SUMS(true, false);
  else if (cz) FPE_BATCH_SUMS(false, true);
  else FPE_BATCH_SUMS(false, false);
#undef FPE_BATCH_SUMS
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return FPE_OK;
}

}  // namespace fpe

// ---------------------------------------------------------------------------
// Evaluation without any allocation (fpe_eval_noalloc)
//
// Some callers cannot allocate device memory when they evaluate: a process
// whose device-memory budget is fixed at start-up, a latency-bound loop that
// must not pay cudaMalloc's cost and implicit device synchronisation, or a
// host program that hands the library only the buffers it owns.  For them the
// per-call scratch of fpe_eval comes from the file-scope array below instead
// of the handle: at most kNoAllocMaxPoints points per call.  Every GPU that
// loads this library holds the array until the process exits, and all calls on
// all handles share it, so calls that overlap on the GPU race.
// ---------------------------------------------------------------------------

namespace fpe {

constexpr int64_t kNoAllocMaxPoints = 32768;
constexpr int64_t kNoAllocExtra = kNoAllocMaxPoints + 1024;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaLo = 0;
constexpr size_t kNaHi = kNaLo + align256(kNoAllocMaxPoints * sizeof(long long));
constexpr size_t kNaKl = kNaHi + align256(kNoAllocMaxPoints * sizeof(long long));
constexpr size_t kNaN = kNaKl + align256(kNoAllocMaxPoints * sizeof(long long));
constexpr size_t kNaKey = kNaN + align256(kNoAllocMaxPoints * sizeof(double));
constexpr size_t kNaRec = kNaKey + align256(2 * kNoAllocMaxPoints * sizeof(uint32_t));  // keys, ranks
constexpr size_t kNaLong = kNaRec + align256(kNoAllocMaxPoints * sizeof(PointRec));
constexpr size_t kNaNg = kNaLong + align256(kNoAllocMaxPoints * sizeof(int32_t));
constexpr size_t kNaGb = kNaNg + align256(kNoAllocMaxPoints * sizeof(int32_t));
constexpr size_t kNaOwner = kNaGb + align256(kNoAllocMaxPoints * sizeof(int32_t));
constexpr size_t kNaGroup = kNaOwner + align256(kNoAllocExtra * sizeof(int32_t));
constexpr size_t kNaVal = kNaGroup + align256(kNoAllocExtra * sizeof(int32_t));
constexpr size_t kNaCarry = kNaVal + align256((kNoAllocMaxPoints + kNoAllocExtra) * sizeof(xdd));
constexpr size_t kNaBins = kNaCarry + align256((kNoAllocMaxPoints + kNoAllocExtra) * sizeof(xdd));
constexpr size_t kNoAllocBytes =
    kNaBins + align256((2 * kNumBins + kNumCounters + kNumBins / kScanTile) * sizeof(uint32_t));
// the figure fpe.h states for the built-in scratch (9,429,248 bytes, about 9.0 MiB)
static_assert(kNoAllocBytes == 9429248, "fpe.h states the size of the built-in scratch: update it with this layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (host code must not use the array's name as an address).
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64] = {nullptr};

static fpe_status noalloc_scratch(int dev, unsigned char **out) {
  if (dev < 0 || dev >= 64) {
    set_error("fpe_eval_noalloc: device ordinal out of range");
    return FPE_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = (unsigned char *)g_noalloc_addr[dev];
  return FPE_OK;
}

}  // namespace fpe

extern "C" fpe_status fpe_eval_noalloc(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n,
                                       fpe_xc64 *out, int32_t *nterms, int32_t *bits_lost, void *cuda_stream) {
  using namespace fpe;
  if (!P || (P->flags & FPE_HOST_ONLY)) {
    set_error("fpe_eval_noalloc: NULL handle or a FPE_HOST_ONLY handle");
    return FPE_ERR_INVALID_ARG;
  }
  if (n < 0 || n > kNoAllocMaxPoints) {
    set_error("fpe_eval_noalloc: n must be in [0, " + std::to_string(kNoAllocMaxPoints) +
              "] (the size of the built-in scratch); use fpe_eval for more points");
    return FPE_ERR_INVALID_ARG;
  }
  if (n > 0 && (!z_re || !out)) {
    set_error("fpe_eval_noalloc: NULL point or output pointer");
    return FPE_ERR_INVALID_ARG;
  }
  if (n == 0) return FPE_OK;
  // the handle's device must be current before its symbol address is looked up
  // (and cached under that device): check both calls
  int prev = -1;
  cudaError_t de = cudaGetDevice(&prev);
  if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
  if (prev != P->device && (de = cudaSetDevice(P->device)) != cudaSuccess) return cuda_fail(de, "cudaSetDevice");
  unsigned char *base = nullptr;
  fpe_status s = noalloc_scratch(P->device, &base);
  if (s == FPE_OK) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Workspace w;  // a view into the built-in scratch; nothing is allocated or freed
    w.cap = kNoAllocMaxPoints;
    w.extra_cap = kNoAllocExtra;
    w.lo = (long long *)(base + kNaLo);
    w.hi = (long long *)(base + kNaHi);
    w.kl = (long long *)(base + kNaKl);
    w.N = (double *)(base + kNaN);
    w.key = (uint32_t *)(base + kNaKey);
    w.rec = (PointRec *)(base + kNaRec);
    w.long_list = (int32_t *)(base + kNaLong);
    w.long_ngroups = (int32_t *)(base + kNaNg);
    w.long_gbase = (int32_t *)(base + kNaGb);
    w.extra_owner = (int32_t *)(base + kNaOwner);
    w.extra_group = (int32_t *)(base + kNaGroup);
    w.group_val = base + kNaVal;
    w.group_carry = base + kNaCarry;
    w.bins = (uint32_t *)(base + kNaBins);
    const int ni = (int)n;
    const int nb = (ni + 255) / 256;
    const bool cz = z_im != nullptr, cc = P->complex_coef;
    // the histogram must start at zero (cursors and counters are written by k_scan_bins)
    cudaError_t e = cudaMemsetAsync(w.bins, 0, kNumBins * sizeof(uint32_t), st);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "cudaMemsetAsync");
    } else {
      if (cz)
        k_locate<true><<<nb, 256, 0, st>>>(P->dev, ni, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, 0);
      else
        k_locate<false><<<nb, 256, 0, st>>>(P->dev, ni, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, 0);
      launch_scan_bins(w.bins, kNumBins, st);
      if (cz)
        k_scatter<true><<<nb, 256, 0, st>>>(P->dev, ni, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, w.rec,
                                            w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner,
                                            w.extra_group, (int)w.extra_cap, P->d_status, P->tune.long_window,
                                            P->tune.group_span(), kNumBins);
      else
        k_scatter<false><<<nb, 256, 0, st>>>(P->dev, ni, z_re, z_im, w.lo, w.hi, w.kl, w.N, w.key, w.key + w.cap, w.bins, w.rec,
                                             w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner,
                                             w.extra_group, (int)w.extra_cap, P->d_status, P->tune.long_window,
                                             P->tune.group_span(), kNumBins);
      const int cap = (int)w.cap, xcap = (int)w.extra_cap;
      const bool acc = P->dev.accurate != 0;
#define FPE_NOALLOC_SUMS(CCv, CZv, ACCv, F32v)                                                                 \
  do {                                                                                                         \
    k_sum_short<CCv, CZv, ACCv, F32v, false>                                                                   \
        <<<(ni + 127) / 128, 128, 0, st>>>(P->dev, nullptr, ni, w.rec, out, nterms, bits_lost,                 \
                                           P->tune.long_window, w.bins + 2 * kNumBins, w.key);                 \
    if (!ACCv && !F32v)                                                                                        \
      k_resum<CCv, CZv, false><<<num_sms() * 6, 128, 0, st>>>(P->dev, nullptr, w.rec, w.bins + 2 * kNumBins,   \
                                                              w.key, out, nterms, bits_lost);                  \
    k_sum_groups<CCv, CZv, ACCv, F32v><<<num_sms() * kSumBlocksPerSm, 128, 0, st>>>(                           \
        P->dev, w.rec, w.long_list, w.long_ngroups, w.long_gbase, w.extra_owner, w.extra_group,                \
        w.bins + 2 * kNumBins, cap, xcap, (xdd *)w.group_val, (xdd *)w.group_carry);                          \
    k_finalize_long<<<num_sms() * 2, 128, 0, st>>>(P->dev, w.rec, w.long_list, w.long_ngroups, w.long_gbase,   \
                                                   w.bins + 2 * kNumBins, cap, (const xdd *)w.group_val,       \
                                                   (const xdd *)w.group_carry, out, nterms, bits_lost);        \
  } while (0)
      const bool f32 = P->dev.fp32 != 0;
      if (cc && cz) {
        if (f32) FPE_NOALLOC_SUMS(true, true, false, true);
        else if (acc) FPE_NOALLOC_SUMS(true, true, true, false);
        else FPE_NOALLOC_SUMS(true, true, false, false);
      } else if (cc) {
        if (f32) FPE_NOALLOC_SUMS(true, false, false, true);
        else if (acc) FPE_NOALLOC_SUMS(true, false, true, false);
        else FPE_NOALLOC_SUMS(true, false, false, false);
      } else if (cz) {
        if (f32) FPE_NOALLOC_SUMS(false, true, false, true);
        else if (acc) FPE_NOALLOC_SUMS(false, true, true, false);
        else FPE_NOALLOC_SUMS(false, true, false, false);
      } else {
        if (f32) FPE_NOALLOC_SUMS(false, false, false, true);
        else if (acc) FPE_NOALLOC_SUMS(false, false, true, false);
        else FPE_NOALLOC_SUMS(false, false, false, false);
      }
#undef FPE_NOALLOC_SUMS
      e = cudaGetLastError();
      if (e != cudaSuccess) s = cuda_fail(e, "fpe_eval_noalloc launch");
    }
  }
  if (prev >= 0 && prev != P->device) cudaSetDevice(prev);
  return s;
}
