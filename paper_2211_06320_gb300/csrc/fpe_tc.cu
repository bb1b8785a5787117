// Window sums of Algorithm A_p (Q_lambda(z) = sum of a_k z^k over
// G_p ∩ [l, r], eq. reducedQlambda) on the tensor cores, for the long windows
// of FP64 evaluations.
//
// The FP64 pipe of this GPU retires about 1.8 lane-FMA per cycle per SM; its
// bf16 tensor cores (mma.sync, fp32 accumulation) about 1000 multiply-adds.
// A window sum over points that share a coefficient window is a dense
// contraction, so it is moved there with every product exact:
//
//   Blocks.  The window is cut into blocks of 32 terms on a grid fixed by the
//   piece's first index k0.  For block m (terms k = k0 + 32 m + i) and point z,
//     C_m = sum_i b_k w^i,  w = 2^beta z  (b_k = a_k 2^-rho(k) on the piece),
//   and the window sum is sum_m C_m W^m with W = w^32.
//
//   Tilt.  The points of a tile (up to 64, bucketed by mu = log2|w|) share a
//   real tilt tau = 2^c with c near their mu: A'_{m,i} = b_k tau^i and
//   Z'_i = u^i with u = w / tau, so A' Z' = b_k w^i, |u| is close to 1 and the
//   products are balanced (the largest |A'| times the largest |Z'| is within
//   2^(62 |mu - c|) of the block's largest term).
//
//   Slices.  Each component of A' (per block) and of Z' (per point) is a
//   69-bit fixed-point number relative to a power of two above its block's or
//   point's largest component, written as ten balanced base-128 digits d_0..d_9
//   (|d| <= 64, exact in bf16).  A digit product is at most 2^12 in
//   magnitude, a 64-long dot product of digits at most 2^18, and the at most
//   ten digit pairs with the same s + s' = t add up below 2^22: fp32
//   accumulation is exact, and adding 1.5 2^23 reads an accumulator back as
//   an integer.  Pairs with t <= 9 are kept (55 of 100); the dropped ones and
//   the truncation leave an error below 2^-66 per product relative to the
//   scales.
//
//   Combination.  The ten integer accumulators of each (block, point) are
//   joined into a 128-bit integer; the blocks of a work item are combined by
//   Horner's scheme in 64-bit mantissas (xh) on the integer pipe, and the work
//   items of a tile in 128-bit ones (xint).
//
// Error per window: below 2^-53.5 times S(z) for tiles with 31 |mu - c| <= 2,
// which the planner enforces (other tiles go back to the FP64 kernels).
//
// MMA layout (tcgen05.mma, kind::f16, M = 128, K = 16 per instruction,
// operands in shared memory, fp32 accumulators in tensor memory): the 128
// rows of A are the tile's 128 points, each row one digit slice of the point's
// Z' over the contraction index kappa = the 32 terms' (real, imaginary)
// powers (K = 64, four k-steps).  B stacks, for a sub-tile of 8 blocks, the
// digit slices sa = 0..9 of A': row 16 sa + 2j + c is block j's real row
// (c = 0) or imaginary row (c = 1) of slice sa,
//   real row (A'_re | -A'_im),  imaginary row (A'_im | A'_re),
// so that out_re = sum_i (A'_re Z'_re - A'_im Z'_im) and
// out_im = sum_i (A'_im Z'_re + A'_re Z'_im).  One MMA takes Z' slice s as A
// and the first N_s = 16 (10 - s) rows of B (the slices sa with s + sa <= 9)
// into the accumulator columns 16 (s + sa) + 2j + c: each column block
// t = s + sa collects exactly the digit pairs of its diagonal, ten MMAs per
// k-step instead of one per pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "fpe_device.cuh"
#include "fpe_internal.h"
#include "fpe_tc05.cuh"
#include "fpe_tc_arith.cuh"

namespace fpe {

namespace {

constexpr int kTK = 2 * kTB;                 // contraction length (re, im per term)
constexpr int kSub = 8;                      // blocks per MMA sub-tile
constexpr int kTcN = 2 * kSub;               // MMA columns: block j's real row 2j, imaginary row 2j + 1
constexpr int kTcEpiWarps = 16;              // warps 0..15 write B's digits and read the accumulators
constexpr int kTcWarps = kTcEpiWarps + 1;    // warp 16 issues the MMAs
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kTcMmaWarp = kTcEpiWarps;
constexpr int kTcPerPoint = kTcEpiWarps / 4; // epilogue threads per point (warps w, w + 4, ... share TMEM lanes)
constexpr int kTcBlkPerThr = kSub / kTcPerPoint;  // blocks of a sub-tile per epilogue thread (2)
static_assert(kTcPoints == 128, "one tile is the M = 128 rows of the MMA");
static_assert(kTK * 2 == 128, "one operand row is 128 bytes: one 128-byte swizzle row");
constexpr double kTcTiltBits = 2.0;          // max 31 |mu - c| over a group's points
// A group takes the bins whose first point lies in a range of kTcGroupSpan
// bucketed positions, so it holds about that many points plus part of a bin:
// a span a little below the tile size lets most groups fill one tile instead
// of spilling a few points into a nearly empty second one.
constexpr int kTcGroupSpan = 112;
constexpr uint32_t kTcPollLimit = 1u << 22;  // polls of an mbarrier before a wait gives up
// every kTcFold sub-tiles a thread folds its 64-bit Horner value into a 128-bit
// one (times W^(8 kTcFold)), so no 64-bit chain is longer than 4 kTcFold steps
constexpr int kTcFold = 16;

struct TcTile {
  int32_t start, count;  // bucketed positions [start, start + count)
  int32_t piece;
  int32_t ok;            // 1: summed here; 0: empty, or handed back to the FP64 kernels
  int64_t mlo;           // first block, counted from the piece's first index
  int64_t nblk;          // blocks covering the union of the tile's windows
  double c;              // tilt exponent
};

// Per tile point, computed once by k_tc_pre: W^(2^k) for k = 0..3 (W = w^32)
// and W^(8 kTcFold), which combine blocks, and Z's scale exponent eq.
struct TcPoint {
  xint W[4];   // W, W^2, W^4, W^8
  xint Wf;     // W^(8 kTcFold): between two folds
  int eq;
  int pad[3];
};

// Per tile: tau^i = tm[i] 2^te[i] for i < 32 (the tilt of A'), 1 / tau and
// tau^32 in 128-bit mantissas (for u = w / tau and W = u^32 tau^32).
struct TcTau {
  unsigned long long tm[kTB];
  int te[kTB];
  xint inv, tau32;
};

// K-major operands with the 128-byte swizzle: a row (one point of A, one
// output row of B) is 128 bytes, the 16-byte chunk c of row r at position
// c ^ (r & 7), eight rows to a 1024-byte atom.  Byte offset of element
// (row r, kappa) in one slice:
__host__ __device__ __forceinline__ int tc_swz(int r, int kappa) {
  return r * 128 + ((((kappa >> 3) ^ (r & 7))) << 4) + ((kappa & 7) << 1);
}
constexpr int kASlice = kTcPoints * 128;           // 16 KB: one slice of A (the tile's Z' digits)
constexpr int kBSlice = kTcN * 128;                // 2 KB: one slice of B (a sub-tile's A' digits)
constexpr int kBBuf = kSl * kBSlice;               // B buffer: the ten slices (160 rows)
constexpr int kZBytes = kSl * kASlice;             // one tile's Z' image (160 KB), as laid out in shared memory

// shared memory of k_tc_sum (offsets from a 1024-byte aligned base)
constexpr int kSmA = 0;                                 // A: 10 slices
constexpr int kSmB = kSmA + kZBytes;                    // B: two buffers of 10 slices
constexpr int kSmW1 = kSmB + 2 * kBBuf;                 // per point W and W^8 (xh), the final exchange
constexpr int kSmW8 = kSmW1 + kTcPoints * (int)sizeof(xh);
constexpr int kSmHx = kSmW8 + kTcPoints * (int)sizeof(xh);  // (kTcPerPoint - 1) values per point
constexpr int kSmTm = kSmHx + (kTcPerPoint - 1) * kTcPoints * (int)sizeof(xh);  // tau^i mantissas
constexpr int kSmTe = kSmTm + kTB * 8;                      // and exponents
constexpr int kSmEq = kSmTe + kTB * 4;                      // Z' scale exponent per point
constexpr int kSmEr = kSmEq + kTcPoints * 4;                // A' scale exponent per block, two buffers
constexpr int kSmBar = kSmEr + 2 * kSub * 4;                // mbarriers: MMA done (2), Z' loaded
constexpr int kSmMisc = kSmBar + 3 * 8;                     // TMEM address, item, tile, abort flag
constexpr int kSmEnd = kSmMisc + 16;
constexpr int kTcSmemBytes = kSmEnd + 1024;                 // + slack for the 1024-byte alignment
static_assert(kSmBar % 8 == 0, "mbarriers are 8-byte aligned");
static_assert(kTcSmemBytes <= 232448, "within the 227 KB of shared memory a block may use");
constexpr uint32_t kTmemCols = 512;          // two buffers of 10 accumulators x 16 columns (320 used)
constexpr int kTmemBuf = kAcc * kTcN;        // columns per buffer

// xor-shuffle of an xint across the warp
__device__ __forceinline__ xint shfl_xint_tc(const xint &v, int m) {
  auto sh = [m](unsigned long long x) { return __shfl_xor_sync(0xffffffffu, x, m); };
  xint r;
  r.x = ((u128)sh((unsigned long long)(v.x >> 64)) << 64) | sh((unsigned long long)v.x);
  r.y = ((u128)sh((unsigned long long)(v.y >> 64)) << 64) | sh((unsigned long long)v.y);
  r.sx = __shfl_xor_sync(0xffffffffu, v.sx, m);
  r.sy = __shfl_xor_sync(0xffffffffu, v.sy, m);
  r.e = (long long)sh((unsigned long long)v.e);
  return r;
}

__device__ __forceinline__ double point_lambda(double zr, double zi) {
  const int f = frexp_exp(fmax(fabs(zr), fabs(zi)));
  const double xr = scale2(zr, -f), xi = scale2(zi, -f);
  return (double)f + 0.5 * log2(fma(xr, xr, xi * xi));
}

__device__ __forceinline__ void tc_write_diag(const DevPoly &P, const PointRec &r, const fpe_xc64 &o,
                                              int32_t *nterms, int32_t *bits_lost) {
  if (nterms) nterms[r.orig] = P.gcount[r.hi + 1] - P.gcount[r.lo];
  if (bits_lost) {
    int bl = 0;
    if (o.re != 0.0 || o.im != 0.0) {
      const double c = ceil(r.N) - (double)o.e;
      bl = c > 0.0 ? (int)fmin(c, 2.0e9) : 0;
    }
    bits_lost[r.orig] = bl;
  }
}


}  // namespace

// ---------------------------------------------------------------------------
// groups and tiles.  The bucketed points of tensor-core piece r occupy
// [s_r, s_r+1); group q of the piece holds the whole bins whose first point
// lies in [s_r + S q, s_r + S (q + 1)) (S = kTcGroupSpan), so a group has
// about S points, or one bin with more.  A group's tilt, the union of its points' windows and
// its work-item boundaries are computed over all its points, and its points
// are cut into tiles of kTcPoints in bucketed order.  Which point of a group
// lands in which tile depends on the scatter's atomics, but nothing a point's
// value depends on does (group boundaries follow from bin counts alone, and
// every MMA column is one point's): results are reproducible bit for bit.
// ---------------------------------------------------------------------------
struct TcGroup {
  int32_t start, count;  // bucketed positions of its points
  int32_t piece;
  int32_t ok;            // 1: tensor cores; 0: empty, or handed back to the FP64 kernels
  int64_t mlo, nblk;     // block range (blocks of kTB terms from the piece's first index)
  double c;              // tilt exponent
};

// the first bin boundary of piece r at or after position x (bins are
// contiguous; bins[nbins + b] is the start of bin b, which the scatter
// leaves in place: it places each point by its rank within the bin)
__device__ __forceinline__ int tc_snap(const uint32_t *bins, int nbins, int r, int x, int s_end) {
  const int b0 = kNumBins + r * kTcBinsPerPiece;
  int a = 0, b = kTcBinsPerPiece;  // find the smallest i with start(b0 + i) >= x
  while (a < b) {
    const int m = (a + b) >> 1;
    if ((int)bins[nbins + b0 + m] >= x)
      b = m;
    else
      a = m + 1;
  }
  return a < kTcBinsPerPiece ? min((int)bins[nbins + b0 + a], s_end) : s_end;
}

// one warp per group: bounds, spread check, tilt, block range
__global__ void k_tc_groups(DevPoly P, PointRec *__restrict__ rec, const uint32_t *__restrict__ bins, int nbins,
                            uint32_t *cnt, TcGroup *__restrict__ groups, int groups_max, long long long_window,
                            long long span, int32_t *__restrict__ long_list, int32_t *__restrict__ long_ngroups,
                            int32_t *__restrict__ long_gbase, int32_t *__restrict__ extra_owner,
                            int32_t *__restrict__ extra_group, int extra_cap) {
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (gw >= groups_max) return;
  int s[kTcMaxPieces + 1];
#pragma unroll
  for (int q = 0; q <= kTcMaxPieces; ++q) s[q] = (int)cnt[kCntTcStart + q];
  int r = -1, lg = 0, cum = 0;
  for (int q = 0; q < P.n_tc && q < kTcMaxPieces; ++q) {
    const int ng = (s[q + 1] - s[q] + kTcGroupSpan - 1) / kTcGroupSpan;
    if (r < 0 && gw < cum + ng) {
      r = q;
      lg = gw - cum;
    }
    cum += ng;
  }
  TcGroup G;
  G.start = G.count = G.piece = G.ok = 0;
  G.mlo = G.nblk = 0;
  G.c = 0.0;
  if (r < 0) {
    if (lane == 0) groups[gw] = G;
    return;
  }
  const int x0 = s[r] + kTcGroupSpan * lg, x1 = x0 + kTcGroupSpan;
  const int start = tc_snap(bins, nbins, r, x0, s[r + 1]);
  const int end = x1 >= s[r + 1] ? s[r + 1] : tc_snap(bins, nbins, r, x1, s[r + 1]);
  const int count = end - start;
  if (count <= 0) {
    if (lane == 0) groups[gw] = G;
    return;
  }
  const int j = P.tc_piece[r];
  const int beta = P.piece_beta[j];
  const long long k0 = P.piece_k0[j];
  double mumin = 1e300, mumax = -1e300;
  long long lomin = LLONG_MAX, himax = LLONG_MIN;
  for (int p = lane; p < count; p += 32) {
    const PointRec q = rec[start + p];
    const double mu = point_lambda(q.zr, q.zi) + (double)beta;
    mumin = fmin(mumin, mu);
    mumax = fmax(mumax, mu);
    lomin = min(lomin, q.lo);
    himax = max(himax, q.hi);
  }
  for (int o = 16; o >= 1; o >>= 1) {
    mumin = fmin(mumin, __shfl_xor_sync(0xffffffffu, mumin, o));
    mumax = fmax(mumax, __shfl_xor_sync(0xffffffffu, mumax, o));
    lomin = min(lomin, (long long)__shfl_xor_sync(0xffffffffu, lomin, o));
    himax = max(himax, (long long)__shfl_xor_sync(0xffffffffu, himax, o));
  }
  G.start = start;
  G.count = count;
  G.piece = j;
  if (31.0 * 0.5 * (mumax - mumin) > kTcTiltBits) {
    // too wide for one tilt: hand the points back to the FP64 kernels
    if (lane == 0) atomicAdd(&cnt[kCntTcRejected], (uint32_t)count);
    for (int p = lane; p < count; p += 32) {
      const int pos = start + p;
      rec[pos].flags = 0;
      const long long L = rec[pos].hi - rec[pos].lo + 1;
      if (L > long_window)
        list_long_window(L, span, (uint32_t)pos, cnt, long_list, long_ngroups, long_gbase, extra_owner,
                         extra_group, extra_cap);
    }
    if (lane == 0) groups[gw] = G;
    return;
  }
  G.ok = 1;
  G.mlo = (lomin - k0) / kTB;
  G.nblk = (himax - k0) / kTB - G.mlo + 1;
  G.c = 0.5 * (mumin + mumax);
  if (lane == 0) groups[gw] = G;
}

// ---------------------------------------------------------------------------
// plan, in three launches: (a) per group its tile count, with the blocks of
// all tiles and the points summed into 64-bit totals; (b) one block: blocks
// per work item (about kTcItemsPerSm items per SM, each at least
// kTcMinChunk blocks) and the scans of tiles and items over the groups;
// (c) per group its tiles, their first items and each item's tile.
// ---------------------------------------------------------------------------
struct TcPlanAcc {
  unsigned long long blocks, points;
};

__device__ __forceinline__ int tc_ntiles(const TcGroup &G) {
  return G.ok ? (G.count + kTcPoints - 1) / kTcPoints : 0;
}

__global__ void __launch_bounds__(256) k_tc_plan_a(const TcGroup *__restrict__ groups, int gm,
                                                   int32_t *__restrict__ g_nt, TcPlanAcc *acc) {
  __shared__ unsigned long long sb[8], sp[8];
  const int g = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long blocks = 0, pts = 0;
  if (g < gm) {
    const TcGroup G = groups[g];
    const int nt = tc_ntiles(G);
    g_nt[g] = nt;
    if (nt) {
      blocks = (unsigned long long)nt * (unsigned long long)G.nblk;
      pts = (unsigned long long)G.count;
    }
  }
  for (int o = 16; o >= 1; o >>= 1) {
    blocks += __shfl_xor_sync(0xffffffffu, blocks, o);
    pts += __shfl_xor_sync(0xffffffffu, pts, o);
  }
  if (lane == 0) {
    sb[wid] = blocks;
    sp[wid] = pts;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tb = 0, tp = 0;
    for (int i = 0; i < 8; ++i) {
      tb += sb[i];
      tp += sp[i];
    }
    if (tb) atomicAdd(&acc->blocks, tb);
    if (tp) atomicAdd(&acc->points, tp);
  }
}

__global__ void __launch_bounds__(1024) k_tc_plan_b(const TcGroup *__restrict__ groups, int gm,
                                                    const int32_t *__restrict__ g_nt, const TcPlanAcc *acc,
                                                    int32_t *__restrict__ g_tile0, int32_t *__restrict__ g_item0,
                                                    uint32_t *cnt, int nsms) {
  __shared__ uint32_t pt[1024], pi[1024];
  __shared__ unsigned long long red[1024];
  const int t = threadIdx.x;
  const int per = (gm + 1023) / 1024;
  const unsigned long long target = (unsigned long long)nsms * kTcItemsPerSm;
  long long chunk = (long long)((acc->blocks + target - 1) / target);
  chunk = std::max<long long>(chunk, kTcMinChunk);
  chunk = (chunk + kSub - 1) / kSub * kSub;
  uint32_t ntl = 0, nit = 0;
  unsigned long long sub = 0;
  const int g0 = min(gm, t * per), g1 = min(gm, (t + 1) * per);
  for (int g = g0; g < g1; ++g) {
    const int nt = g_nt[g];
    if (!nt) continue;
    const long long nblk = groups[g].nblk;
    const long long ipt = (nblk + chunk - 1) / chunk;
    ntl += (uint32_t)nt;
    nit += (uint32_t)(nt * ipt);
    sub += (unsigned long long)nt * (unsigned long long)((ipt - 1) * (chunk / kSub) +
                                                         (nblk - (ipt - 1) * chunk + kSub - 1) / kSub);
  }
  pt[t] = ntl;
  pi[t] = nit;
  red[t] = sub;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scans of tiles and items
    const uint32_t a = t >= o ? pt[t - o] : 0u, b = t >= o ? pi[t - o] : 0u;
    __syncthreads();
    pt[t] += a;
    pi[t] += b;
    __syncthreads();
  }
  for (int o = 512; o >= 1; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  uint32_t tt = pt[t] - ntl, it = pi[t] - nit;
  for (int g = g0; g < g1; ++g) {
    const int nt = g_nt[g];
    g_tile0[g] = (int32_t)tt;
    g_item0[g] = (int32_t)it;
    if (!nt) continue;
    const long long ipt = (groups[g].nblk + chunk - 1) / chunk;
    tt += (uint32_t)nt;
    it += (uint32_t)(nt * ipt);
  }
  if (t == 0) {
    cnt[kCntTcItems] = pi[1023];
    cnt[kCntTcChunk] = (uint32_t)chunk;
    cnt[kCntTcWork] = 0;
    cnt[kCntTcTiles] = pt[1023];
    cnt[kCntTcPoints] = (uint32_t)acc->points;
    cnt[kCntTcSubtiles] = (uint32_t)min(red[0], 0xffffffffull);
  }
}

__global__ void __launch_bounds__(256) k_tc_plan_c(const TcGroup *__restrict__ groups, int gm,
                                                   const int32_t *__restrict__ g_nt,
                                                   const int32_t *__restrict__ g_tile0,
                                                   const int32_t *__restrict__ g_item0, const uint32_t *cnt,
                                                   TcTile *__restrict__ tiles, int tiles_max,
                                                   int32_t *__restrict__ item_base, int32_t *__restrict__ item_tile) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const long long chunk = (long long)cnt[kCntTcChunk];
  const int ntile_total = (int)cnt[kCntTcTiles];
  const int nitem_total = (int)cnt[kCntTcItems];
  if (tid < gm && g_nt[tid]) {
    const TcGroup G = groups[tid];
    const int nt = g_nt[tid];
    const int ipt = (int)((G.nblk + chunk - 1) / chunk);
    for (int lt = 0; lt < nt; ++lt) {
      const int tt = g_tile0[tid] + lt, it = g_item0[tid] + lt * ipt;
      TcTile T;
      T.start = G.start + kTcPoints * lt;
      T.count = min(kTcPoints, G.count - kTcPoints * lt);
      T.piece = G.piece;
      T.ok = 1;
      T.mlo = G.mlo;
      T.nblk = G.nblk;
      T.c = G.c;
      tiles[tt] = T;
      item_base[tt] = it;
      for (int c = 0; c < ipt; ++c) item_tile[it + c] = tt;
    }
  }
  for (int i = ntile_total + tid; i < tiles_max; i += nthr) {  // unused tiles
    TcTile T;
    T.start = T.count = T.piece = T.ok = 0;
    T.mlo = T.nblk = 0;
    T.c = 0.0;
    tiles[i] = T;
    item_base[i + 1] = nitem_total;
  }
  if (tid == 0) item_base[ntile_total] = nitem_total;
}

// ---------------------------------------------------------------------------
// per tile, one warp: tau = 2^c (as tmant 2^tf, tmant in [0.5, 1)), lane i
// tau^i, lane 0 1 / tau, lane 1 tau^32 (all lanes at once)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_tau(const TcTile *__restrict__ tiles, TcTau *__restrict__ taus,
                                                const uint32_t *cnt) {
  const int ntiles = (int)cnt[kCntTcTiles], lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nw) {
    const double tau = exp2(tiles[t].c);
    const int tf = frexp_exp(tau);
    const double tmant = scale2(tau, -tf);
    xint ti = xint_norm((u128)1 << 126, 0, 0, 0, 0);
    if (lane > 0) {
      ti = xint_pow_unit(tmant, 0.0, lane);
      ti.e += (long long)tf * lane;
    }
    taus[t].tm[lane] = (unsigned long long)(ti.x >> 63);  // in [2^63, 2^64)
    taus[t].te[lane] = (int)(ti.e - 63);
    if (lane == 0) {
      xint inv = recip_xint(tmant, 0.0);
      inv.e -= tf;
      taus[t].inv = inv;
    } else if (lane == 1) {
      xint t32 = xint_pow_unit(tmant, 0.0, kTB);
      t32.e += (long long)tf * kTB;
      taus[t].tau32 = t32;
    }
  }
}

// per tile point (four threads, eight powers each): u = w / tau, and the Z' slices of u^i
// (i < 32) written to global memory in exactly the layout k_tc_sum copies
// into shared memory as the MMA's A operand: per slice, the point's row of
// 128 bytes (kappa = i for the real part of u^i, 32 + i for the imaginary
// part), as 16-byte chunks at their swizzled positions (eight powers at a
// time, one chunk per slice and component); W^(2^k) = (u^32 tau^32)^(2^k),
// W^(8 kTcFold), and Z's scale exponent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_tc_pre(DevPoly P, const PointRec *__restrict__ rec,
                                                const TcTile *__restrict__ tiles, TcPoint *__restrict__ pts,
                                                const TcTau *__restrict__ taus, unsigned char *__restrict__ zglob,
                                                const uint32_t *cnt) {
  // a unit is 32 points of a tile (lane = point) times the four groups of eight
  // powers (warp g: u^(8g) .. u^(8g + 7)); warp 0 also forms the points' W
  const int ntiles = (int)cnt[kCntTcTiles], lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  for (int unit = blockIdx.x; unit < 4 * ntiles; unit += gridDim.x) {
    const int t = unit >> 2, p = 32 * (unit & 3) + lane;
    const TcTile T = tiles[t];
    const bool valid = p < T.count;
    const xint zero = xint_norm(0, 0, 0, 0, 0);
    xint u = zero;
    xh uh = xh_norm(0, 0, 0, 0, 0), cur = uh;
    int eQ = 1;
    if (valid) {
      const PointRec r = rec[T.start + p];
      u = xint_mul(xint_from_dd2(r.zr, 0.0, r.zi, 0.0, P.piece_beta[T.piece]), taus[t].inv);
      uh = xh_from_xint(u);
      // every |component of u^i| (i < 32) is at most |u|^31 <= 2^(eQ - 1); |u| is
      // near 1, so log2|u| in FP32 (error far below the 1e-3 / 31 margin) suffices:
      // |u| = sqrt(mx^2 + my^2) 2^e with mx = X 2^-126 (X the magnitude, top bit at 126)
      const float mx = (float)(unsigned long long)(u.x >> 64) * 0x1p-62f;
      const float my = (float)(unsigned long long)(u.y >> 64) * 0x1p-62f;
      const float l = 0.5f * log2f(fmaf(mx, mx, my * my)) + (float)u.e;
      eQ = max(0, (int)ceilf(31.0f * l + 1e-3f)) + 1;
      // u^(8g) by squarings (u^24 = u^16 u^8)
      cur = xh_norm(1ull << 63, 0, 0, 0, 0);  // 1
      if (g > 0) {
        const xh u2 = xh_mul(uh, uh), u4 = xh_mul(u2, u2), u8 = xh_mul(u4, u4);
        cur = g == 1 ? u8 : xh_mul(u8, u8);
        if (g == 3) cur = xh_mul(cur, u8);
      }
    }
    // powers u^i in 64-bit mantissas: u^i comes from products whose exponents add
    // up to i, each truncating at 2^-63 of its value, so u^31 is within 2^-58 of
    // its value relative to itself
    unsigned char *zt = zglob + (size_t)t * kZBytes;
    uint32_t wr[kSl][4], wi[kSl][4];  // bf16 pairs of powers 8g + 2q, 8g + 2q + 1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t xr[2][kSl], xi[2][kSl];
      DigitSign sr[2], si[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if ((q | h) != 0 && valid) cur = xh_mul(cur, uh);
        // x 2^(e - 63) 2^(70 - eq) = x 2^-sh with eq = eQ + 1: fixed point below
        // 2^69 (components <= 2^(eQ - 1))
        const int sh = eQ + 1 + 63 - 70 - (int)cur.e;
        bchunks70(valid ? shift_to70((u128)cur.x, sh) : (u128)0, xr[h]);
        bchunks70(valid ? shift_to70((u128)cur.y, sh) : (u128)0, xi[h]);
        sr[h] = digit_sign((uint32_t)cur.sx);
        si[h] = digit_sign((uint32_t)cur.sy);
      }
#pragma unroll
      for (int s = 0; s < kSl; ++s) {
        wr[s][q] = bf16_pair(xr[0][s], sr[0], xr[1][s], sr[1]);
        wi[s][q] = bf16_pair(xi[0][s], si[0], xi[1][s], si[1]);
      }
    }
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
      *reinterpret_cast<uint4 *>(zt + s * kASlice + tc_swz(p, 8 * g)) =
          make_uint4(wr[s][0], wr[s][1], wr[s][2], wr[s][3]);
      *reinterpret_cast<uint4 *>(zt + s * kASlice + tc_swz(p, kTB + 8 * g)) =
          make_uint4(wi[s][0], wi[s][1], wi[s][2], wi[s][3]);
    }
    if (g == 0) {
      TcPoint o;
      xint W = zero;
      if (valid) {  // W = u^32 tau^32 = w^32 from the 128-bit u: the block weights W^g and
        // the Horner multipliers must not inherit the 64-bit powers' error
        xint u32 = u;
        for (int k = 0; k < 5; ++k) u32 = xint_sqr(u32);
        W = xint_mul(u32, taus[t].tau32);
      }
      o.W[0] = W;
      for (int k = 1; k < 4; ++k) o.W[k] = xint_sqr(o.W[k - 1]);
      o.Wf = o.W[3];
      for (int q = 1; (1 << q) <= kTcFold; ++q) o.Wf = xint_sqr(o.Wf);
      o.eq = eQ + 1;  // Z' = F 2^(eq - 70)
      o.pad[0] = o.pad[1] = o.pad[2] = 0;
      pts[(size_t)t * kTcPoints + p] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// the window sums on the tensor cores.  One persistent CTA per SM (17 warps) takes work
// items (a tile and a run of at most `chunk` blocks) from a counter.  Per
// item, the tile's Z' image (the A operand, 160 KB) arrives by ten bulk
// copies on an mbarrier; then, sub-tile by sub-tile of 8 blocks from the top
// down, in a two-stage pipeline:
//   warps 0-15 write B's digits for sub-tile s (one component of one term per
//     thread) into one of two buffers, then read the accumulators of sub-tile s + 1;
//   warp 16 (converged, one elected lane) issues the 40 MMAs of sub-tile s
//     (10 Z' slices x 4 k-steps, each against the stacked A' slices) into one
//     of two sets of ten TMEM accumulators and commits them to that set's
//     mbarrier.
// Thread w 32 + l of warps 0-15 is TMEM lane 32 (w % 4) + l, i.e. point
// p = 32 (w % 4) + l, and takes blocks 2 h, 2 h + 1 (h = w / 4) of each
// sub-tile: it joins each block's ten fp32 accumulators (real and imaginary
// columns, one per diagonal) into 128-bit integers and runs Horner's scheme
// over its sub-tiles in 64-bit mantissas, H <- H W^8 + C_1 W + C_0, folded
// every kTcFold sub-tiles into a 128-bit value.  At the end of the item the
// four parts of each point are joined, V = A_0 + W^2 (A_1 + W^2 (A_2 + W^2 A_3)),
// and the value goes to the item's slot.  Every mbarrier wait is bounded; a wait
// that gives up sets FPE_ERR_TIMEOUT's status bit and the CTA stops.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_sum(DevPoly P, const TcTile *__restrict__ tiles, const TcPoint *__restrict__ pts,
             const TcTau *__restrict__ taus, const unsigned char *__restrict__ zglob,
             const int32_t *__restrict__ item_base, const int32_t *__restrict__ item_tile, uint32_t *cnt,
             xint *__restrict__ slots, int32_t *status) {
  using namespace tc05;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // swizzle atoms: 1024-aligned
  xh *sW1 = reinterpret_cast<xh *>(sm + kSmW1);
  xh *sW8 = reinterpret_cast<xh *>(sm + kSmW8), *sHx = reinterpret_cast<xh *>(sm + kSmHx);
  unsigned long long *sTm = reinterpret_cast<unsigned long long *>(sm + kSmTm);
  int *sTe = reinterpret_cast<int *>(sm + kSmTe), *sEq = reinterpret_cast<int *>(sm + kSmEq);
  int *sEr = reinterpret_cast<int *>(sm + kSmEr);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kSmBar);  // [0], [1]: MMAs done per buffer; [2]: Z' loaded
  volatile int *misc = reinterpret_cast<volatile int *>(sm + kSmMisc);  // TMEM address, item, tile
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool mma_thread = tid == kTcMmaWarp * 32;  // issues the bulk copies
  const uint32_t nitems = *(volatile uint32_t *)&cnt[kCntTcItems];
  const long long chunk = (long long)*(volatile uint32_t *)&cnt[kCntTcChunk];
  const xint zero = xint_norm(0, 0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    fence_mbar_init();
  }
  if (wid == kTcMmaWarp) {
    tmem_alloc(reinterpret_cast<uint32_t *>(sm + kSmMisc), kTmemCols);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = (uint32_t)misc[0];
  const uint32_t aaddr = smem_u32(sm + kSmA), baddr = smem_u32(sm + kSmB);
  const uint64_t adesc0 = desc_sw128_kmajor(aaddr);
  uint32_t ph_mma[2] = {0u, 0u}, ph_z = 0u;  // parity of the next phase each mbarrier completes
  int abort = 0;                             // this thread saw a wait give up
  // epilogue thread: point p, blocks 2 h, 2 h + 1 of each sub-tile
  const int p = 32 * (wid & 3) + lane, h = (wid >> 2) & 3;

  while (true) {
    if (tid == 0) {
      const uint32_t it = atomicAdd(&cnt[kCntTcWork], 1u);
      misc[1] = (int)it;
      misc[2] = it < nitems ? item_tile[it] : -1;
    }
    __syncthreads();
    const int item = misc[1], t = misc[2];
    if (t < 0) break;
    const TcTile T = tiles[t];
    const int j = T.piece;
    const long long k0 = P.piece_k0[j], k1 = (long long)P.piece_k0[j + 1] - 1;
    const long long mb = T.mlo + (long long)(item - item_base[t]) * chunk;
    const long long me = min((long long)(T.mlo + T.nblk), mb + chunk);
    const int nsub = (int)((me - mb + kSub - 1) / kSub);
    const TcPoint *tp = pts + (size_t)t * kTcPoints;

    // ---- setup: the Z' image by bulk copies; tau^i and the points' multipliers
    if (mma_thread) {
      mbar_arrive_expect_tx(&bar[2], (uint32_t)kZBytes);
      const unsigned char *src = zglob + (size_t)t * kZBytes;
#pragma unroll 1
      for (int s = 0; s < kSl; ++s) bulk_g2s(sm + kSmA + s * kASlice, src + s * kASlice, kASlice, &bar[2]);
    }
    if (tid < kTcPoints) {
      const bool v = tid < T.count;
      sW1[tid] = xh_from_xint(v ? tp[tid].W[0] : zero);
      sW8[tid] = xh_from_xint(v ? tp[tid].W[3] : zero);
      sEq[tid] = v ? tp[tid].eq : 1;
    } else if (tid < kTcPoints + kTB) {
      sTm[tid - kTcPoints] = taus[t].tm[tid - kTcPoints];
      sTe[tid - kTcPoints] = taus[t].te[tid - kTcPoints];
    }
    if (!mbar_wait(&bar[2], ph_z, kTcPollLimit)) {
      abort = 1;
      atomicOr(status, kStatusTimeout);
    }
    ph_z ^= 1u;
    if (__syncthreads_or(abort)) break;

    // ---- sub-tiles of 8 blocks, from the top down
    const xh w1 = sW1[p], w8 = sW8[p];
    const int eqp = sEq[p];
    xh H = xh_norm(0, 0, 0, 0, 0);
    xint Acc = zero;  // the folded 128-bit value
    int e_prev[kTcBlkPerThr] = {0, 0}, e_cur[kTcBlkPerThr] = {0, 0};
    // coefficient of this thread's term in block mb + 8 ts + (wid % 8) (0 outside the item or the piece)
    auto load_b = [&](int ts_) -> double2 {
      const long long m = mb + (long long)kSub * ts_ + (wid & (kSub - 1));
      const long long k = k0 + kTB * m + lane;
      double2 c = make_double2(0.0, 0.0);
      if (ts_ >= 0 && m < me && k <= k1) {
        if (P.complex_coef)
          c = __ldg(reinterpret_cast<const double2 *>(P.b) + k);
        else
          c.x = __ldg(P.b + k);
      }
      return c;
    };
    double2 bnext = load_b(nsub - 1);
    for (int it = 0; it <= nsub; ++it) {
      const int ts = nsub - 1 - it;  // the sub-tile whose digits and MMAs this iteration makes
      const int buf = it & 1;
      if (it < nsub && wid < kTcEpiWarps) {  // B's digits: warp w takes block w % 8, component w / 8, lane = term
        const int jb = wid & (kSub - 1), comp = wid >> 3;
        const double br = bnext.x, bi = bnext.y;
        bnext = load_b(ts - 1);  // in flight during this sub-tile
        const unsigned long long tmi = sTm[lane];
        const int tei = sTe[lane];
        // both components' products give the block's scale; the digits are this thread's component's
        u128 pr = 0, pi = 0;
        int er_ = 0, ei_ = 0, top = INT_MIN;
        auto prod = [&](double x, u128 &pp, int &E) {
          const unsigned long long bits = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
          if (bits == 0) return;
          const int ex = (int)(bits >> 52);
          const unsigned long long mm = ex ? ((bits & 0xfffffffffffffull) | 0x10000000000000ull)
                                           : (bits & 0xfffffffffffffull);
          pp = (u128)mm * tmi;
          E = (ex ? ex : 1) - 1075 + tei;
          top = max(top, 127 - clz128(pp) + E);
        };
        prod(br, pr, er_);
        prod(bi, pi, ei_);
        for (int o = 16; o >= 1; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
        const int eR = top == INT_MIN ? 0 : top + 2;  // every |component| < 2^(eR - 1): below 2^69 in F
        const u128 pc = comp ? pi : pr;
        const u128 F = pc ? shift_to70(pc, eR - 70 - (comp ? ei_ : er_)) : (u128)0;
        uint32_t x[kSl];
        bchunks70(F, x);
        const DigitSign sg = digit_sign((uint32_t)((comp ? bi : br) < 0.0));
        // in slice s, real row 16 s + 2 jb = (A'_re | -A'_im) and imaginary row
        // 16 s + 2 jb + 1 = (A'_im | A'_re): a real part goes to (real row, kappa i)
        // and (imaginary row, 32 + i), an imaginary part negated to (real row, 32 + i)
        // and as it is to (imaginary row, i).  A slice is 16 rows, two whole 8-row
        // swizzle atoms, so the row's swizzle phase does not depend on s.
        const int o1 = comp ? tc_swz(2 * jb, kTB + lane) : tc_swz(2 * jb, lane);
        const int o2 = comp ? tc_swz(2 * jb + 1, lane) : tc_swz(2 * jb + 1, kTB + lane);
        const uint16_t flip = comp ? 0x8000u : 0u;
        unsigned char *Bb = sm + kSmB + buf * kBBuf;
#pragma unroll
        for (int s = 0; s < kSl; ++s) {
          const uint16_t d = (uint16_t)(tc_fbits(fmaf(tc_bitsf(x[s]), sg.s, sg.k)) >> 16);  // bf16 of the digit
          *reinterpret_cast<uint16_t *>(Bb + s * kBSlice + o1) = d ^ flip;
          *reinterpret_cast<uint16_t *>(Bb + s * kBSlice + o2) = d;
        }
        if (lane == 0 && comp == 0) sEr[buf * kSub + jb] = eR;
      }
      // B (written by the generic proxy) becomes visible to the tensor core; the
      // epilogue's TMEM reads of this buffer's previous use are ordered before
      // the MMAs that overwrite it
      fence_proxy_async_smem();
      fence_before_sync();
      if (__syncthreads_or(abort)) break;
      fence_after_sync();
      if (it < nsub) {
#pragma unroll
        for (int q = 0; q < kTcBlkPerThr; ++q) e_cur[q] = sEr[buf * kSub + kTcBlkPerThr * h + q];
        if (wid == kTcMmaWarp) {  // the MMA warp, converged; one elected lane issues
          // for Z' slice s: D[cols 16 s ..] (+)= A(slice s) B(rows 0 .. N_s - 1)^T, N_s as above;
          // the first MMA (s = 0, k-step 0) covers every column and starts the sums
          const uint32_t dcol = tbase + (uint32_t)(buf * kTmemBuf);
          const uint64_t bdesc0 = desc_sw128_kmajor(baddr + (uint32_t)(buf * kBBuf));
          if (elect_one()) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
              for (int sz = 0; sz < kSl; ++sz) {
                const int ncol = kTcN * (kAcc - sz);
                const uint32_t d = dcol + (uint32_t)(kTcN * sz);
                const uint64_t a = adesc0 + (uint64_t)((sz * kASlice + 32 * ks) >> 4);
                const uint64_t b = bdesc0 + (uint64_t)((32 * ks) >> 4);
                if (ks == 0 && sz == 0)
                  mma_bf16_set(d, a, b, idesc_bf16_f32(kTcPoints, ncol));
                else
                  mma_bf16_acc(d, a, b, idesc_bf16_f32(kTcPoints, ncol));
              }
            }
            mma_commit(&bar[buf]);
          }
          __syncwarp();
        }
      }
      if (it > 0 && wid < kTcEpiWarps) {  // epilogue of the previous sub-tile
        const int pb = (it - 1) & 1;
        const bool ok = mbar_wait(&bar[pb], ph_mma[pb], kTcPollLimit);
        ph_mma[pb] ^= 1u;
        if (!ok) {
          abort = 1;
          atomicOr(status, kStatusTimeout);
        } else {
          fence_after_sync();
          // block 2 h + jj of the sub-tile: columns 16 t + 2 (2 h + jj) + (0 real, 1 imaginary)
          const uint32_t ta = tbase + ((uint32_t)(32 * (wid & 3)) << 16) + (uint32_t)(pb * kTmemBuf + 4 * h);
          const long long m0 = mb + (long long)kSub * (ts + 1);  // the previous sub-tile's first block
          xh C[kTcBlkPerThr];
#pragma unroll
          for (int jj = kTcBlkPerThr - 1; jj >= 0; --jj) {
            uint32_t v[kAcc][2];
#pragma unroll
            for (int tt = 0; tt < kAcc; ++tt) tmem_ld2(ta + (uint32_t)(kTcN * tt + 2 * jj), v[tt]);
            tmem_ld_wait();
            C[jj] = xh_norm(0, 0, 0, 0, 0);
            if (m0 + kTcBlkPerThr * h + jj < me && p < T.count) {
              float ar[kAcc], ai[kAcc];
#pragma unroll
              for (int tt = 0; tt < kAcc; ++tt) {
                ar[tt] = __uint_as_float(v[tt][0]);
                ai[tt] = __uint_as_float(v[tt][1]);
              }
              u128 xr, xi;
              int sr, si;
              join_vals(ar, xr, sr);
              join_vals(ai, xi, si);
              // A' = F 2^(eR - 70), Z' = F 2^(eq - 70), and the kept pairs are
              // 128^9 X: C = X 2^(eR + eq - 77) = X 2^(e - 126) with e = eR + eq + 49
              C[jj] = xh_from128(xr, sr, xi, si, 49 + (long long)e_prev[jj] + eqp);
            }
          }
          // H (relative to block 2 h of the sub-tile above, 8 blocks up) <- H W^8 + C_1 W + C_0:
          // the two products are independent
          xh T1 = C[1];
          if (T1.x || T1.y) T1 = xh_mul(T1, w1);
          if (H.x || H.y) H = xh_mul(H, w8);
          H = xh_add(xh_add(H, T1), C[0]);
          if ((ts + 1) % kTcFold == 0) {  // fold: Acc = Acc W^(8 kTcFold) + H (the folds are that far apart)
            if (Acc.x || Acc.y) Acc = xint_mul(Acc, tp[p].Wf);
            Acc = xint_add(Acc, xint_from_xh(H));
            H = xh_norm(0, 0, 0, 0, 0);
          }
        }
        fence_before_sync();
      }
#pragma unroll
      for (int q = 0; q < kTcBlkPerThr; ++q) e_prev[q] = e_cur[q];
    }
    if (__syncthreads_or(abort)) break;
    // ---- V = A_0 + W^2 (A_1 + W^2 (A_2 + W^2 A_3)) per point (the last sub-tile, 0,
    // ended with a fold), into the item's slot
    if (wid < kTcEpiWarps && h > 0) sHx[(h - 1) * kTcPoints + p] = xh_from_xint(Acc);
    __syncthreads();
    if (wid < kTcEpiWarps && h == 0 && p < T.count) {
      const xint W2 = tp[p].W[1];
      xint V = xint_from_xh(sHx[(kTcPerPoint - 2) * kTcPoints + p]);
      for (int q = kTcPerPoint - 2; q >= 0; --q) {
        if (V.x || V.y) V = xint_mul(V, W2);
        V = xint_add(V, q > 0 ? xint_from_xh(sHx[(q - 1) * kTcPoints + p]) : Acc);
      }
      slots[(size_t)item * kTcPoints + p] = V;
    }
    __syncthreads();  // shared memory is reused by the next item
  }
  fence_before_sync();
  __syncthreads();
  if (wid == kTcMmaWarp) tmem_dealloc(tbase, kTmemCols);
}

// b^n (n >= 1) by binary powering
__device__ __forceinline__ xint xint_pow_x(xint b, long long n) {
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

// Per tile point: the sum over the tile's items, item c starting c chunks of
// blocks after the first, i.e. sum_c V_c (W^chunk)^c; then z^(kb + v)
// 2^rho(kb) with kb the first block's index, and the point's output.
// W^chunk = (W^8)^(chunk / 8) from the powers k_tc_pre stored.  Tiles of at
// most kFinOneLaneItems items take one thread per point (L = 1: most tiles
// have one item, and the power z^(kb + v) is the thread's main work);
// longer ones eight (L = 8, blocks of half a tile): threads q < 7 take a contiguous seventh of the
// items by Horner in W^chunk and scale it by (W^chunk)^(its first item),
// thread 7 computes z^(kb + v) meanwhile, and the parts are added by
// shuffles.  Each launch skips the other's tiles.
constexpr int kFinOneLaneItems = 4;
// A block takes PPB points of a tile (kTcPoints / PPB blocks per tile).
template <int L, int PPB>
__global__ void __launch_bounds__(L * PPB)
    k_tc_finalize(DevPoly P, const PointRec *__restrict__ rec, const TcTile *__restrict__ tiles,
                  const TcPoint *__restrict__ pts, const int32_t *__restrict__ item_base, const uint32_t *cnt,
                  const xint *__restrict__ slots, fpe_xc64 *__restrict__ out, int32_t *nterms,
                  int32_t *bits_lost) {
  constexpr int kParts = kTcPoints / PPB;
  const int ntiles = (int)cnt[kCntTcTiles], q = threadIdx.x % L;
  constexpr int qpow = L - 1;            // the thread that computes z^(kb + v)
  constexpr int nh = L > 1 ? L - 1 : 1;  // threads that take items
  for (int u = blockIdx.x; u < ntiles * kParts; u += gridDim.x) {
    const int t = u / kParts, p = (u % kParts) * PPB + (int)threadIdx.x / L;
    const int base = item_base[t], nit = item_base[t + 1] - base;
    if ((L == 1) != (nit <= kFinOneLaneItems)) continue;  // the other launch's tile
    const TcTile T = tiles[t];
    const bool valid = p < T.count;
    const long long chunk = (long long)cnt[kCntTcChunk];
    const int j = T.piece;
    const xint zero = xint_norm(0, 0, 0, 0, 0);
    PointRec r;
    r.zr = r.zi = 0.0;
    if (valid) r = rec[T.start + p];
    const int f = valid ? frexp_exp(fmax(fabs(r.zr), fabs(r.zi))) : 0;
    const int per = (nit + nh - 1) / nh;
    const int c0 = q * per, c1 = q < nh ? min(nit, c0 + per) : c0;
    xint V = zero, zp = zero;
    if (valid) {
      if (c0 < c1) {
        xint Wc = zero;
        if (nit > 1) {  // W^chunk = w^(32 chunk); k_tc_plan_b makes chunk a multiple of kSub = 8,
                        // the power of z below only guards that invariant
          if (chunk % 8 == 0) {
            Wc = xint_pow_x(pts[(size_t)t * kTcPoints + p].W[3], chunk / 8);
          } else {
            Wc = xint_pow_z(r.zr, r.zi, kTB * chunk, f);
            Wc.e += (long long)kTB * chunk * P.piece_beta[j];
          }
        }
        for (int c = c1 - 1; c >= c0; --c) {
          if (V.x || V.y) V = xint_mul(V, Wc);
          V = xint_add(V, slots[(size_t)(base + c) * kTcPoints + p]);
        }
        if (c0 > 0 && (V.x || V.y)) V = xint_mul(V, xint_pow_x(Wc, c0));  // times Wc^c0
      }
      if (q == qpow) {  // z^(kb + v), kb = k0 + 32 mlo
        const long long kb = P.piece_k0[j] + kTB * T.mlo;
        zp = xint_pow_z(r.zr, r.zi, kb + P.v, f);
        zp.e += P.piece_rho0[j] + (long long)P.piece_beta[j] * (kb - P.piece_k0[j]);
      }
    }
    if (L > 1) {  // add the L parts (lanes L p .. L p + L - 1 of one warp)
      for (int o = 1; o < L; o <<= 1) {
        const xint w = shfl_xint_tc(V, o);
        V = xint_add(V, w);
      }
      zp = shfl_xint_tc(zp, qpow);  // thread 0 gets thread qpow's power
    }
    if (valid && q == 0) {
      if (V.x || V.y) V = xint_mul(V, zp);
      const fpe_xc64 o = xc64_from_xint(V);
      out[r.orig] = o;
      tc_write_diag(P, r, o, nterms, bits_lost);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int tc_num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

static int64_t tc_groups_max(int64_t n) { return (n + kTcGroupSpan - 1) / kTcGroupSpan + kTcMaxPieces; }
static int64_t tc_tiles_max(int64_t n) { return (n + kTcPoints - 1) / kTcPoints + tc_groups_max(n); }
static int64_t tc_items_cap(int64_t n) { return tc_tiles_max(n) + (int64_t)tc_num_sms() * kTcItemsPerSm; }

// The path's planning costs about ten launches whatever the size, which a
// call with few points does not recover (measured: d = 1000 with 10^4
// points, 0.50 ms with the path against 0.39 without), so by default it
// runs on calls of at least tc_min_points points; an explicit
// fpe_set_tensor_path applies to every call.
bool tc_enabled(const fpe_poly_s *P, bool complex_points, int64_t n) {
  (void)complex_points;
  return P->dev.n_tc > 0 && !P->dev.fp32 && !P->dev.accurate && P->tune.tc_min_window > 0 &&
         n >= P->tune.tc_min_points;
}

void free_tc_workspace(Workspace &w) {
  void *ptrs[] = {w.tc_tiles, w.tc_item_base, w.tc_slots, w.tc_points, w.tc_item_tile, w.tc_taus, w.tc_z,
                  w.tc_groups, w.tc_plan};
  for (void *a : ptrs)
    if (a) cudaFree(a);
  w.tc_tiles = nullptr;
  w.tc_item_base = nullptr;
  w.tc_slots = nullptr;
  w.tc_points = nullptr;
  w.tc_item_tile = nullptr;
  w.tc_taus = nullptr;
  w.tc_z = nullptr;
  w.tc_groups = nullptr;
  w.tc_plan = nullptr;
  w.tc_cap = 0;
}

fpe_status ensure_tc_workspace(fpe_poly_s *P, int64_t n) {
  Workspace &w = P->ws;
  const int64_t cap = std::max<int64_t>(n, 1024);
  if (w.tc_cap >= cap && w.tc_tiles) return FPE_OK;
  free_tc_workspace(w);
  const int64_t tm = tc_tiles_max(cap), ic = tc_items_cap(cap);
  cudaError_t e = cudaMalloc(&w.tc_tiles, tm * sizeof(TcTile));
  if (e == cudaSuccess) e = cudaMalloc((void **)&w.tc_item_base, (tm + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&w.tc_slots, (size_t)ic * kTcPoints * sizeof(xint));
  if (e == cudaSuccess) e = cudaMalloc(&w.tc_points, (size_t)tm * kTcPoints * sizeof(TcPoint));
  if (e == cudaSuccess) e = cudaMalloc((void **)&w.tc_item_tile, (size_t)ic * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&w.tc_taus, (size_t)tm * sizeof(TcTau));
  if (e == cudaSuccess) e = cudaMalloc(&w.tc_z, (size_t)tm * kZBytes);
  if (e == cudaSuccess) e = cudaMalloc(&w.tc_groups, (size_t)tc_groups_max(cap) * sizeof(TcGroup));
  // plan scratch: the 64-bit totals, then per group its tiles, first tile and first item
  if (e == cudaSuccess)
    e = cudaMalloc(&w.tc_plan, sizeof(TcPlanAcc) + 3 * (size_t)tc_groups_max(cap) * sizeof(int32_t));
  if (e != cudaSuccess) {
    free_tc_workspace(w);
    return cuda_fail(e, "cudaMalloc(tensor-core workspace)");
  }
  w.tc_cap = cap;
  return FPE_OK;
}


// the kernels' dynamic shared memory above the default 48 KB, once per device
static fpe_status tc_set_smem_attrs() {
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_sum, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tensor-core kernels)");
    attr_set[dev] = true;
  }
  return FPE_OK;
}

fpe_status launch_tc_groups(fpe_poly_s *P, int n, cudaStream_t st) {
  fpe_status s = tc_set_smem_attrs();
  if (s != FPE_OK) return s;
  Workspace &w = P->ws;
  uint32_t *cnt = w.bins + 2 * w.nbins;
  const int gm = (int)tc_groups_max(n);
  {
    ProfScope ps("k_tc_groups", st);
    k_tc_groups<<<(gm + 7) / 8, 256, 0, st>>>(P->dev, w.rec, w.bins, w.nbins, cnt, (TcGroup *)w.tc_groups, gm,
                                              P->tune.long_window, P->tune.group_span(), w.long_list,
                                              w.long_ngroups, w.long_gbase, w.extra_owner, w.extra_group,
                                              (int)w.extra_cap);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "tensor-core groups launch");
}

fpe_status launch_tc_plan(fpe_poly_s *P, int n, cudaStream_t st) {
  Workspace &w = P->ws;
  uint32_t *cnt = w.bins + 2 * w.nbins;
  const int tm = (int)tc_tiles_max(n), gm = (int)tc_groups_max(n);
  {
    ProfScope ps("k_tc_plan", st, 3);  // k_tc_plan_a, _b, _c
    TcPlanAcc *acc = (TcPlanAcc *)w.tc_plan;
    int32_t *g_nt = (int32_t *)(acc + 1), *g_tile0 = g_nt + gm, *g_item0 = g_tile0 + gm;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(TcPlanAcc), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(plan)");
    k_tc_plan_a<<<(gm + 255) / 256, 256, 0, st>>>((const TcGroup *)w.tc_groups, gm, g_nt, acc);
    k_tc_plan_b<<<1, 1024, 0, st>>>((const TcGroup *)w.tc_groups, gm, g_nt, acc, g_tile0, g_item0, cnt,
                                    tc_num_sms());
    k_tc_plan_c<<<(gm + 255) / 256, 256, 0, st>>>((const TcGroup *)w.tc_groups, gm, g_nt, g_tile0, g_item0, cnt,
                                                  (TcTile *)w.tc_tiles, tm, w.tc_item_base, w.tc_item_tile);
  }
  {
    ProfScope ps("k_tc_pre", st, 2);  // k_tc_tau, k_tc_pre
    k_tc_tau<<<std::min((tm + 7) / 8, tc_num_sms() * 8), 256, 0, st>>>((const TcTile *)w.tc_tiles,
                                                                       (TcTau *)w.tc_taus, cnt);
    k_tc_pre<<<std::min(4 * tm, tc_num_sms() * 16), 128, 0, st>>>(P->dev, w.rec, (const TcTile *)w.tc_tiles,
                                                                    (TcPoint *)w.tc_points,
                                                                    (const TcTau *)w.tc_taus, (unsigned char *)w.tc_z, cnt);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "tensor-core plan launch");
}

fpe_status launch_tc_sums(fpe_poly_s *P, int n, fpe_xc64 *out, int32_t *nterms, int32_t *bits_lost,
                          cudaStream_t st) {
  Workspace &w = P->ws;
  uint32_t *cnt = w.bins + 2 * w.nbins;
  const int tm = (int)tc_tiles_max(n);
  fpe_status s = tc_set_smem_attrs();
  if (s != FPE_OK) return s;
  {
    ProfScope ps("k_tc_sum", st);
    k_tc_sum<<<tc_num_sms(), kTcThreads, kTcSmemBytes, st>>>(
        P->dev, (const TcTile *)w.tc_tiles, (const TcPoint *)w.tc_points, (const TcTau *)w.tc_taus,
        (const unsigned char *)w.tc_z, w.tc_item_base, w.tc_item_tile, cnt, (xint *)w.tc_slots, P->d_status);
  }
  {
    ProfScope ps("k_tc_finalize", st, 2);  // eight- and one-thread launches
    k_tc_finalize<8, kTcPoints / 2><<<std::min(2 * tm, tc_num_sms() * 4), 8 * (kTcPoints / 2), 0, st>>>(
        P->dev, w.rec, (const TcTile *)w.tc_tiles, (const TcPoint *)w.tc_points, w.tc_item_base, cnt,
        (const xint *)w.tc_slots, out, nterms, bits_lost);
    k_tc_finalize<1, kTcPoints><<<std::min(tm, tc_num_sms() * 16), kTcPoints, 0, st>>>(
        P->dev, w.rec, (const TcTile *)w.tc_tiles, (const TcPoint *)w.tc_points, w.tc_item_base, cnt,
        (const xint *)w.tc_slots, out, nterms, bits_lost);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "tensor-core sum launch");
}

}  // namespace fpe

extern "C" fpe_status fpe_tensor_stats(fpe_poly_t P, int64_t *stats, int n, void *cuda_stream) {
  using namespace fpe;
  if (!P || !stats || n < 6) {
    set_error("fpe_tensor_stats: NULL handle or output, or n < 6");
    return FPE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) stats[i] = 0;
  if (!P->ws.bins || P->ws.nbins <= kNumBins) return FPE_OK;  // the last evaluation did not use the path
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != P->device) cudaSetDevice(P->device);
  uint32_t c[kNumCounters];
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemcpyAsync(c, P->ws.bins + 2 * P->ws.nbins, sizeof c, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (prev >= 0 && prev != P->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "fpe_tensor_stats");
  stats[0] = c[kCntTcPoints];
  stats[1] = c[kCntTcTiles];
  stats[2] = c[kCntTcItems];
  stats[3] = c[kCntTcSubtiles];
  stats[4] = c[kCntTcChunk];
  stats[5] = c[kCntTcRejected];
  return FPE_OK;
}

extern "C" fpe_status fpe_cert_stats(fpe_poly_t P, int64_t *stats, int n, void *cuda_stream) {
  using namespace fpe;
  if (!P || !stats || n < 1) {
    set_error("fpe_cert_stats: NULL handle or output, or n < 1");
    return FPE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i) stats[i] = 0;
  if (!P->ws.bins || P->dev.fp32 || P->dev.accurate) return FPE_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != P->device) cudaSetDevice(P->device);
  uint32_t c[kNumCounters];
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemcpyAsync(c, P->ws.bins + 2 * P->ws.nbins, sizeof c, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (prev >= 0 && prev != P->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "fpe_cert_stats");
  stats[0] = c[kCntResum];
  return FPE_OK;
}
