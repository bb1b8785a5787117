// Host preconditioning of Algorithm A_p (its preconditioning part, §5.1): exact integer scales,
// the concave cover of k -> s(a_k), the good set G_p, and the device layout of
// the coefficients.  Runs once per polynomial; not on the evaluation path.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "fpe_internal.h"

namespace fpe {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error_cstr() { return g_last_error.c_str(); }

fpe_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FPE_ERR_OOM : FPE_ERR_CUDA;
}

typedef __int128 i128;
static const int64_t kNoScale = std::numeric_limits<int64_t>::min();

// ---------------------------------------------------------------------------
// Scales (eq. dsz; eq. sz)
// ---------------------------------------------------------------------------

// frexp exponent: x = m 2^f with |m| in [0.5, 1), so 2^(f-1) <= |x| < 2^f.
static int frexp_exp(double x) {
  int f;
  std::frexp(x, &f);
  return f;
}

// x^2 + y^2 >= 4^f, exactly, given max(|x|, |y|) in [2^(f-1), 2^f).
// Scaled X = |x| 2^-f, Y = |y| 2^-f lie in [0, 1).  The FP64 sum of squares
// is within 2^-51 of the truth; only near 1 is the test redone exactly: if the
// smaller value is below 2^-27 the answer is no (the larger square is at most
// 1 - 2^-52 + 2^-106); otherwise X 2^80 and Y 2^80 are integers below 2^80
// and their squares are summed in three 64-bit limbs.
static bool abs2_ge_pow4(double x, double y, int f) {
  double X = std::ldexp(std::fabs(x), -f), Y = std::ldexp(std::fabs(y), -f);
  double q = X * X + Y * Y;
  if (q > 1.0 + 0x1p-50) return true;
  if (q < 1.0 - 0x1p-50) return false;
  double M = X > Y ? X : Y, m = X > Y ? Y : X;
  if (m < 0x1p-27) return false;
  auto to_int = [](double t) -> unsigned __int128 {
    // t in [2^-27, 1) has 53 significant bits with the lowest at >= 2^-80
    double hi = std::ldexp(t, 80 - 64);  // t 2^16, integer part < 2^16
    double ih = std::floor(hi);
    double rem = std::ldexp(hi - ih, 64);  // exact: < 2^64, integer
    return ((unsigned __int128)(uint64_t)ih << 64) + (unsigned __int128)(uint64_t)rem;
  };
  unsigned __int128 A = to_int(M), B = to_int(m);
  // squares as 3 limbs (base 2^64): a = ah 2^64 + al with ah < 2^16
  uint64_t limb[3] = {0, 0, 0};
  auto add_sq = [&limb](unsigned __int128 a) {
    uint64_t ah = (uint64_t)(a >> 64), al = (uint64_t)a;
    unsigned __int128 ll = (unsigned __int128)al * al;          // at 2^0
    unsigned __int128 lh = (unsigned __int128)al * ah * 2;      // at 2^64, < 2^81
    unsigned __int128 hh = (unsigned __int128)ah * ah;          // at 2^128, < 2^32
    unsigned __int128 c = (unsigned __int128)limb[0] + (uint64_t)ll;
    limb[0] = (uint64_t)c;
    c = (c >> 64) + limb[1] + (uint64_t)(ll >> 64) + (uint64_t)lh;
    limb[1] = (uint64_t)c;
    c = (c >> 64) + limb[2] + (uint64_t)(lh >> 64) + (uint64_t)hh;
    limb[2] = (uint64_t)c;
  };
  add_sq(A);
  add_sq(B);
  // compare with 2^160 = limb[2] == 2^32, lower limbs 0
  return limb[2] >= (1ull << 32);
}

static int64_t scale_of(double re, double im, bool cplx) {
  if (!cplx || im == 0.0) {
    if (re == 0.0) return kNoScale;
    return frexp_exp(re);
  }
  if (re == 0.0) return frexp_exp(im);
  int f = std::max(frexp_exp(re), frexp_exp(im));
  return f + (abs2_ge_pow4(re, im, f) ? 1 : 0);
}

static int bit_length(int64_t n) {
  int b = 0;
  while (n > 0) {
    ++b;
    n >>= 1;
  }
  return b;
}

// round(num / den) for den > 0, halves rounded up
static int64_t round_div(i128 num, i128 den) {
  i128 t = 2 * num + den;
  i128 q = t / (2 * den);
  if ((t % (2 * den)) < 0) q -= 1;  // floor
  return (int64_t)q;
}

// ---------------------------------------------------------------------------
// Device upload helpers
// ---------------------------------------------------------------------------

template <class T>
static fpe_status upload(fpe_poly_s *P, const std::vector<T> &h, const T **dst) {
  if (h.empty()) {
    *dst = nullptr;
    return FPE_OK;
  }
  void *d = nullptr;
  cudaError_t e = cudaMalloc(&d, h.size() * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  P->allocs.push_back(d);
  e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  *dst = (const T *)d;
  return FPE_OK;
}

void free_handle(fpe_poly_s *P) {
  if (!P) return;
  if (P->flags & FPE_HOST_ONLY) {
    if (P->deriv) free_handle(P->deriv);
    delete P;
    return;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  for (void *a : P->allocs) cudaFree(a);
  free_workspace(P->ws);
  if (P->aux) cudaFree(P->aux);
  if (P->d_status) cudaFree(P->d_status);
  if (P->tc_stream) cudaStreamDestroy(P->tc_stream);
  if (P->tc_fork) cudaEventDestroy(P->tc_fork);
  if (P->tc_join) cudaEventDestroy(P->tc_join);
  cudaSetDevice(prev);
  if (P->deriv) free_handle(P->deriv);
  delete P;
}

void free_workspace(Workspace &w) {
  void *ptrs[] = {w.lo,          w.hi,          w.kl,           w.N,          w.key,
                  w.rec,         w.long_list,   w.long_ngroups, w.long_gbase, w.extra_owner,
                  w.extra_group, w.group_val,   w.group_carry,  w.bins,       w.dev_io};
  for (void *a : ptrs)
    if (a) cudaFree(a);
  if (w.host_pinned) cudaFreeHost(w.host_pinned);
  free_tc_workspace(w);
  w = Workspace();
}

// per-point scratch for n points (the bins are allocated separately)
fpe_status alloc_workspace(Workspace &w, int64_t n) {
  const int64_t cap = std::max<int64_t>(n, 1024);
  const int64_t xcap = cap + 1024;  // extra group slots for very long windows
  void **slots[] = {(void **)&w.lo,          (void **)&w.hi,          (void **)&w.kl,
                    (void **)&w.N,           (void **)&w.key,         (void **)&w.rec,
                    (void **)&w.long_list,   (void **)&w.long_ngroups, (void **)&w.long_gbase,
                    (void **)&w.extra_owner, (void **)&w.extra_group, &w.group_val,
                    &w.group_carry};
  for (void **a : slots) {
    if (*a) cudaFree(*a);
    *a = nullptr;
  }
  w.cap = 0;
  w.extra_cap = 0;
  const size_t xval = 40;  // extended double-double value
  const size_t sizes[] = {cap * sizeof(long long), cap * sizeof(long long), cap * sizeof(long long),
                          cap * sizeof(double),    2 * cap * sizeof(uint32_t), cap * sizeof(PointRec),
                          cap * sizeof(int32_t),   cap * sizeof(int32_t),   cap * sizeof(int32_t),
                          xcap * sizeof(int32_t),  xcap * sizeof(int32_t),  (cap + xcap) * xval,
                          (cap + xcap) * xval};
  for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
    cudaError_t e = cudaMalloc(slots[i], sizes[i]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
  }
  w.cap = cap;
  w.extra_cap = xcap;
  return FPE_OK;
}

fpe_status ensure_workspace(fpe_poly_s *P, int64_t n) {
  Workspace &w = P->ws;
  if (w.bins == nullptr) {
    cudaError_t e = cudaMalloc((void **)&w.bins,
                                  (3 * (kNumBins + kTcBins) + kNumCounters) * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(bins)");
  }
  if (n <= w.cap) return FPE_OK;
  return alloc_workspace(w, n);
}

// ---------------------------------------------------------------------------
// Preconditioning
// ---------------------------------------------------------------------------

fpe_status precondition_host(const double *re, const double *im, const int64_t *e2, int64_t n_coef, int p,
                             uint32_t flags, fpe_poly_s **out) {
  if (!out) {
    set_error("fpe_precondition: out is NULL");
    return FPE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!re || n_coef < 1 || n_coef > (int64_t)1 << 30) {
    set_error("fpe_precondition: re is NULL or n_coef out of [1, 2^30]");
    return FPE_ERR_INVALID_ARG;
  }
  if (flags & ~(uint32_t)(FPE_REAL | FPE_WITH_DERIV | FPE_FP32 | FPE_HOST_ONLY | FPE_ACCURATE | FPE_FORCE_DENSE |
                          FPE_FORCE_SPARSE)) {
    set_error("fpe_precondition: unknown flag bits");
    return FPE_ERR_INVALID_ARG;
  }
  const bool fp32 = (flags & FPE_FP32) != 0;
  if (p < 2 || p > 53 || (fp32 && p > 24)) {
    set_error("fpe_precondition: p must be in [2, 53] ([2, 24] with FPE_FP32)");
    return FPE_ERR_INVALID_ARG;
  }
  if ((flags & FPE_FORCE_DENSE) && (flags & FPE_FORCE_SPARSE)) {
    set_error("fpe_precondition: FPE_FORCE_DENSE and FPE_FORCE_SPARSE together");
    return FPE_ERR_INVALID_ARG;
  }
  if (fp32 && (flags & FPE_ACCURATE)) {
    set_error("fpe_precondition: FPE_FP32 with FPE_ACCURATE is not available in this build");
    return FPE_ERR_UNSUPPORTED;
  }
  bool cplx = im != nullptr && !(flags & FPE_REAL);
  for (int64_t k = 0; k < n_coef; ++k) {
    if (!std::isfinite(re[k]) || (cplx && !std::isfinite(im[k]))) {
      set_error("fpe_precondition: non-finite coefficient at index " + std::to_string(k));
      return FPE_ERR_NONFINITE;
    }
    if (e2 && (e2[k] > ((int64_t)1 << 40) || e2[k] < -((int64_t)1 << 40))) {
      set_error("fpe_precondition: |e2[k]| must be below 2^40");
      return FPE_ERR_INVALID_ARG;
    }
  }
  if (cplx) {  // real polynomial if every imaginary part is zero (§8.1 detects this case)
    bool any = false;
    for (int64_t k = 0; k < n_coef && !any; ++k) any = im[k] != 0.0;
    cplx = any;
  }

  // scales s(a_k) (eq. dsz), untrimmed
  std::vector<int64_t> s(n_coef);
  int64_t v = -1, d = -1;
  for (int64_t k = 0; k < n_coef; ++k) {
    int64_t sk = scale_of(re[k], cplx ? im[k] : 0.0, cplx);
    if (sk != kNoScale && e2) sk += e2[k];
    s[k] = sk;
    if (sk != kNoScale) {
      if (v < 0) v = k;
      d = k;
    }
  }
  if (d < 0) {
    set_error("fpe_precondition: every coefficient is zero");
    return FPE_ERR_ZERO_POLY;
  }

  const bool host_only = (flags & FPE_HOST_ONLY) != 0;
  fpe_poly_s *P = new fpe_poly_s();
  if (!host_only) cudaGetDevice(&P->device);
  P->p = p;
  P->flags = flags;
  P->n_coef = n_coef;
  P->d = d;
  P->v = v;
  P->complex_coef = cplx;
  const int64_t D = d - v;
  // T = p + s(d) + 3 with s(d) the bit length of the degree (Alg. A_p, eq. threshold)
  P->T = p + (d >= 1 ? bit_length(d) : 0) + 3;
  const int64_t T = P->T;

  // concave cover over the nonzero points (k, s_k): upper hull by a monotone
  // chain in k, which yields the same unique cover as the paper's sorted
  // incremental construction; collinear points are dropped.
  std::vector<int64_t> hk, hs;  // trimmed abscissae
  for (int64_t k = 0; k <= D; ++k) {
    int64_t sk = s[v + k];
    if (sk == kNoScale) continue;
    while (hk.size() >= 2) {
      size_t m = hk.size();
      i128 cross = (i128)(hk[m - 1] - hk[m - 2]) * (sk - hs[m - 2]) - (i128)(hs[m - 1] - hs[m - 2]) * (k - hk[m - 2]);
      if (cross >= 0) {  // middle point on or under the chord: not a strict vertex
        hk.pop_back();
        hs.pop_back();
      } else {
        break;
      }
    }
    hk.push_back(k);
    hs.push_back(sk);
  }
  const int nh = (int)hk.size();
  P->hull_k.resize(nh);
  P->hull_s = hs;
  for (int i = 0; i < nh; ++i) P->hull_k[i] = hk[i] + v;

  // G_p (eq. threshold): s_k >= cover(k) - T, exactly, segment by segment
  P->good.assign(n_coef, 0);
  std::vector<int32_t> gcount(D + 2, 0);
  {
    int seg = 0;
    for (int64_t k = 0; k <= D; ++k) {
      int64_t sk = s[v + k];
      bool g = false;
      if (sk != kNoScale) {
        if (nh == 1) {
          g = true;
        } else {
          while (seg + 1 < nh - 1 && hk[seg + 1] <= k) ++seg;
          i128 dk = hk[seg + 1] - hk[seg], ds = hs[seg + 1] - hs[seg];
          g = (i128)(sk - hs[seg] + T) * dk >= ds * (k - hk[seg]);
        }
      }
      P->good[v + k] = g;
      gcount[k + 1] = gcount[k] + (g ? 1 : 0);
    }
    P->n_good = gcount[D + 1];
  }
  std::vector<int32_t> good_idx;  // for the sparse window sums
  good_idx.reserve(P->n_good);
  for (int64_t k = 0; k <= D; ++k)
    if (P->good[v + k]) good_idx.push_back((int32_t)k);

  // pieces: cut [0, D] at multiples of the piece length and at every vertex
  const int log2_piece = fp32 ? kLog2PieceLenF32 : kLog2PieceLen;
  const int64_t kPieceLen = (int64_t)1 << log2_piece;
  std::vector<int32_t> pk0, pbeta, pdelta, pfirst;
  std::vector<int64_t> prho0;
  {
    std::vector<int64_t> cuts;
    int vi = 1;
    for (int64_t c = 0; c <= D;) {
      cuts.push_back(c);
      int64_t nxt = (c / kPieceLen + 1) * kPieceLen;
      while (vi < nh && hk[vi] <= c) ++vi;
      if (vi < nh && hk[vi] < nxt) nxt = hk[vi];
      c = nxt;
    }
    const int np = (int)cuts.size();
    pk0.resize(np + 1);
    pbeta.resize(np);
    prho0.resize(np);
    pdelta.resize(np);
    int seg = 0;
    for (int j = 0; j < np; ++j) {
      int64_t c = cuts[j];
      pk0[j] = (int32_t)c;
      if (nh == 1 || c >= hk[nh - 1]) {
        pbeta[j] = 0;
        prho0[j] = hs[nh - 1];
        continue;
      }
      while (seg + 1 < nh - 1 && hk[seg + 1] <= c) ++seg;
      i128 dk = hk[seg + 1] - hk[seg], ds = hs[seg + 1] - hs[seg];
      // cover(c) = hs[seg] + ds (c - hk[seg]) / dk, rounded; beta = round(ds / dk)
      prho0[j] = round_div((i128)hs[seg] * dk + ds * (c - hk[seg]), dk);
      int64_t b = round_div(ds, dk);
      if (b > 100000 || b < -100000) b = b > 0 ? 100000 : -100000;
      pbeta[j] = (int32_t)b;
    }
    pk0[np] = (int32_t)(D + 1);
    for (int j = 0; j < np; ++j) {
      int64_t len = pk0[j + 1] - pk0[j];
      pdelta[j] = (j + 1 < np) ? (int32_t)(prho0[j + 1] - prho0[j] - (int64_t)pbeta[j] * len) : 0;
    }
    // Merge runs of pieces into one piece with an integer line rho(k) =
    // rho0 + beta (k - k0) that stays within kMergeDrift bits of every
    // merged piece's own line (at both ends of each, hence all along it;
    // FP64 modes; the FP32 mode merges only exact continuations, to keep
    // its values inside the FP32 range).  A nearly flat cover then becomes
    // one piece instead of being cut every few hundred terms by the rounding
    // of rho0 to integers, and a cover like that of P' (steep over its first
    // few terms, then rising by one bit per doubling of k) one or two: the
    // windows stay inside one piece for the tensor-core sums, and the FP64
    // loops see fewer crossings.  b_k = a_k 2^-rho(k) stays within
    // kMergeDrift bits (kMergeDriftSteep for a nonzero slope: the measured
    // certificates of steep covers, e.g. 1/k!, fared better with shorter
    // pieces) of where the unmerged pieces put it.  For a run starting at
    // piece m the slopes of the next pieces are tried and the one that
    // merges the longest run is kept; rho0 is the middle of the feasible
    // range.
    {
      constexpr int64_t kMergeDrift = 24, kMergeDriftSteep = 8;
      // longest run m..e-1 mergeable with slope b; the feasible rho0 range in [lo_r, hi_r]
      auto run_with = [&](int m, int64_t b, int64_t &lo_r, int64_t &hi_r) {
        const int64_t max_off = fp32 ? 0 : (b == 0 ? kMergeDrift : kMergeDriftSteep);
        lo_r = INT64_MIN / 4;
        hi_r = INT64_MAX / 4;
        int e = m;
        for (; e < np; ++e) {
          int64_t a = lo_r, c = hi_r;
          for (int end = 0; end < 2; ++end) {
            const int64_t k = end ? (int64_t)pk0[e + 1] : (int64_t)pk0[e];
            const int64_t target = end ? prho0[e] + (int64_t)pbeta[e] * (pk0[e + 1] - pk0[e]) : prho0[e];
            const int64_t base = target - b * (k - pk0[m]);  // rho0 that puts the line on target at k
            a = std::max(a, base - max_off);
            c = std::min(c, base + max_off);
          }
          if (a > c) break;
          lo_r = a;
          hi_r = c;
        }
        return e;
      };
      std::vector<int32_t> nk0, nbeta;
      std::vector<int64_t> nrho0;
      for (int m = 0; m < np;) {
        int best_e = m + 1;
        int64_t best_b = pbeta[m], best_lo = prho0[m], best_hi = prho0[m];
        for (int q = m; q < np && q < m + 6; ++q) {
          if (q > m && pbeta[q] == pbeta[q - 1]) continue;
          int64_t lo_r, hi_r;
          const int e = run_with(m, pbeta[q], lo_r, hi_r);
          if (e > best_e || (e == best_e && q == m)) {
            best_e = e;
            best_b = pbeta[q];
            best_lo = lo_r;
            best_hi = hi_r;
          }
        }
        if (best_e == m + 1 && best_b == pbeta[m]) {
          best_lo = best_hi = prho0[m];  // a piece on its own keeps its line
        }
        nk0.push_back(pk0[m]);
        nbeta.push_back((int32_t)best_b);
        nrho0.push_back(best_lo + (best_hi - best_lo) / 2);
        m = best_e;
      }
      const int nm = (int)nk0.size();
      pk0.assign(nk0.begin(), nk0.end());
      pk0.push_back((int32_t)(D + 1));
      pbeta = nbeta;
      prho0 = nrho0;
      pdelta.resize(nm);
      for (int q = 0; q < nm; ++q)  // the exponent jumps between the merged pieces
        pdelta[q] = (q + 1 < nm) ? (int32_t)(prho0[q + 1] - prho0[q] - (int64_t)pbeta[q] * (pk0[q + 1] - pk0[q])) : 0;
    }
    const int npm = (int)pbeta.size();
    int64_t nblk = D / kPieceLen + 1;
    pfirst.resize(nblk + 1);
    int j = 0;
    for (int64_t g = 0; g <= nblk; ++g) {
      int64_t start = g * kPieceLen;
      while (j + 1 < npm && pk0[j + 1] <= start) ++j;
      pfirst[g] = j;
    }
    P->dev.npieces = npm;
    // pieces for the tensor-core window sums: complex FP64 default mode, the
    // longest (merged) pieces of at least kTcMinPieceLen terms
    P->dev.n_tc = 0;
    for (int r = 0; r < kTcMaxPieces; ++r) P->dev.tc_piece[r] = -1;
    if (!fp32 && !(flags & FPE_ACCURATE)) {
      std::vector<std::pair<int64_t, int>> byLen;
      for (int q = 0; q < npm; ++q) {
        const int64_t len = (int64_t)pk0[q + 1] - pk0[q];
        if (len >= kTcMinPieceLen) byLen.push_back({-len, q});
      }
      std::sort(byLen.begin(), byLen.end());
      for (size_t r = 0; r < byLen.size() && r < (size_t)kTcMaxPieces; ++r) P->dev.tc_piece[P->dev.n_tc++] = byLen[r].second;
    }
  }

  // coefficients b_k = a_k 2^-rho(k), trimmed; bad ones zeroed in b
  const int stride = cplx ? 2 : 1;
  std::vector<double> b((D + 1) * stride), bfull((D + 1) * stride);
  std::vector<float> bf;
  {
    int j = 0;
    const int np = P->dev.npieces;
    for (int64_t k = 0; k <= D; ++k) {
      while (j + 1 < np && pk0[j + 1] <= k) ++j;
      int64_t rho = prho0[j] + (int64_t)pbeta[j] * (k - pk0[j]);
      int64_t sh = (e2 ? e2[v + k] : 0) - rho;
      int ish = (int)std::max<int64_t>(-4000, std::min<int64_t>(4000, sh));
      double br = std::ldexp(re[v + k], ish);
      double bi = cplx ? std::ldexp(im[v + k], ish) : 0.0;
      bool g = P->good[v + k] != 0;
      bfull[k * stride] = br;
      b[k * stride] = g ? br : 0.0;
      if (cplx) {
        bfull[k * stride + 1] = bi;
        b[k * stride + 1] = g ? bi : 0.0;
      }
    }
  }

  std::vector<uint64_t> bq;
  std::vector<float> bm;  // FP64 modes: magnitude lower bounds for the rounding-error certificates
  if (fp32) {  // the p-bit representation of the kept coefficients (Thm. equivAlgo's tilde a_k)
    bf.resize(b.size());
    for (size_t i = 0; i < b.size(); ++i) bf[i] = (float)b[i];
  } else {  // integer-pipe copy for the window sums
    bm.resize(D + 1);
    for (int64_t k = 0; k <= D; ++k) bm[k] = coef_mag_lo(b[k * stride], cplx ? b[k * stride + 1] : 0.0);
    bq.resize(b.size());
    for (size_t i = 0; i < b.size(); ++i) {
      bq[i] = qpack(b[i]);
      if (bq[i] == ~(uint64_t)0) {
        set_error("fpe_precondition: a rescaled coefficient is outside the packed exponent range");
        free_handle(P);
        return FPE_ERR_UNSUPPORTED;
      }
    }
  }

  // a_0 for z = 0 (§4.2: P(0) = a_0), normalised
  if (v == 0) {
    double a0r = re[0], a0i = cplx ? im[0] : 0.0;
    int f = frexp_exp(std::fabs(a0r) > std::fabs(a0i) ? a0r : a0i);
    P->dev.a0_re = std::ldexp(a0r, -f);
    P->dev.a0_im = std::ldexp(a0i, -f);
    P->dev.a0_e = f + (e2 ? e2[0] : 0);
  }

  // device arrays
  std::vector<double> dhk(nh), dhs(nh), dsig(nh > 1 ? nh - 1 : 0);
  for (int i = 0; i < nh; ++i) {
    dhk[i] = (double)hk[i];
    dhs[i] = (double)hs[i];
  }
  for (int i = 0; i + 1 < nh; ++i) dsig[i] = (double)(hs[i + 1] - hs[i]) / (double)(hk[i + 1] - hk[i]);

  fpe_status st;
  DevPoly &dp = P->dev;
  if (!host_only) {
    if ((st = upload(P, b, &dp.b)) != FPE_OK || (st = upload(P, bf, &dp.bf)) != FPE_OK ||
        (st = upload(P, bq, &dp.bq)) != FPE_OK || (st = upload(P, bm, &dp.bmag)) != FPE_OK ||
        (st = upload(P, bfull, &dp.b_full)) != FPE_OK ||
        (st = upload(P, pk0, &dp.piece_k0)) != FPE_OK ||
        (st = upload(P, pbeta, &dp.piece_beta)) != FPE_OK ||
        (st = upload(P, pdelta, &dp.piece_delta)) != FPE_OK ||
        (st = upload(P, prho0, &dp.piece_rho0)) != FPE_OK ||
        (st = upload(P, pfirst, &dp.piece_first)) != FPE_OK ||
        (st = upload(P, dhk, &dp.hull_k)) != FPE_OK ||
        (st = upload(P, dhs, &dp.hull_s)) != FPE_OK ||
        (st = upload(P, dsig, &dp.hull_sig)) != FPE_OK ||
        (st = upload(P, gcount, &dp.gcount)) != FPE_OK || (st = upload(P, good_idx, &dp.good_idx)) != FPE_OK) {
      free_handle(P);
      return st;
    }
    cudaError_t e = cudaMalloc((void **)&P->d_status, sizeof(int32_t));
    if (e != cudaSuccess) {
      free_handle(P);
      return cuda_fail(e, "cudaMalloc(status)");
    }
    cudaMemset(P->d_status, 0, sizeof(int32_t));
  }
  dp.D = D;
  dp.v = v;
  dp.T = (double)T;
  dp.n_hull = nh;
  dp.complex_coef = cplx ? 1 : 0;
  dp.fp32 = fp32 ? 1 : 0;
  dp.accurate = (flags & FPE_ACCURATE) ? 1 : 0;
  dp.sparse_mode = (flags & FPE_FORCE_DENSE) ? 1 : ((flags & FPE_FORCE_SPARSE) ? 2 : 0);
  dp.log2_piece = log2_piece;

  // P' (§7.2): coefficients (k+1) a_{k+1}, rounded once, preconditioned separately
  if (flags & FPE_WITH_DERIV) {
    if (d == 0) {
      P->deriv_zero = true;
    } else {
      std::vector<double> dre(d), dim(cplx ? d : 0);
      std::vector<int64_t> de2(e2 ? d : 0);
      for (int64_t k = 0; k < d; ++k) {
        dre[k] = (double)(k + 1) * re[k + 1];
        if (cplx) dim[k] = (double)(k + 1) * im[k + 1];
        if (e2) de2[k] = e2[k + 1];
      }
      fpe_poly_s *Q = nullptr;
      fpe_status ds = precondition_host(dre.data(), cplx ? dim.data() : nullptr, e2 ? de2.data() : nullptr, d, p,
                                        flags & ~(uint32_t)FPE_WITH_DERIV, &Q);
      if (ds == FPE_ERR_ZERO_POLY) {
        P->deriv_zero = true;
      } else if (ds != FPE_OK) {
        free_handle(P);
        return ds;
      } else {
        P->deriv = Q;
      }
    }
  }
  *out = P;
  return FPE_OK;
}

}  // namespace fpe
