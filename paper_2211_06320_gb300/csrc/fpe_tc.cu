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
//   accumulation is exact.  Pairs with t <= 9 are kept (55 of 100); the
//   dropped ones and the truncation leave an error below 2^-66 per product
//   relative to the scales.
//
//   Combination.  The ten integer accumulators of each (block, point) are
//   joined into a 128-bit integer; the blocks of a work item are combined by
//   Horner's scheme in 64-bit mantissas (xh) on the integer pipe, and the work
//   items of a tile in 128-bit ones (xint).
//
// Error per window: below 2^-53.5 times S(z) for tiles with 31 |mu - c| <= 2,
// which the planner enforces (other tiles go back to the FP64 kernels).
//
// MMA layout (m16n8k16, A row-major 16 x 16, B column 16 x 8): the 16 rows of
// A are 8 blocks x (real part, imaginary part) of the output, the 8 columns
// of B are 8 points, and the contraction index kappa runs over the 32 terms'
// (real, imaginary) point powers:
//   out_re = sum_i (A'_re Z'_re - A'_im Z'_im),  out_im = sum_i (A'_im Z'_re + A'_re Z'_im).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "fpe_device.cuh"
#include "fpe_internal.h"
#include "fpe_tc_arith.cuh"

namespace fpe {

namespace {

constexpr int kTK = 2 * kTB;                 // contraction length (re, im per term)
constexpr int kSub = 8;                      // blocks per MMA sub-tile (16 rows)
constexpr int kTcWarps = kTcPoints / 8;      // one warp per 8 points (and per block of a sub-tile)
constexpr int kTcThreads = 32 * kTcWarps;
static_assert(kTcWarps == kSub, "the A' tile is built one block per warp");
constexpr double kTcTiltBits = 2.0;          // max 31 |mu - c| over a group's points

struct TcTile {
  int32_t start, count;  // bucketed positions [start, start + count)
  int32_t piece;
  int32_t ok;            // 1: summed here; 0: empty, or handed back to the FP64 kernels
  int64_t mlo;           // first block, counted from the piece's first index
  int64_t nblk;          // blocks covering the union of the tile's windows
  double c;              // tilt exponent
};

// Per tile point, computed once by k_tc_pre: W^(2^k) for k = 0..3 (W = w^32),
// which combine blocks, and Z's scale exponent eq.
struct TcPoint {
  xint W[4];   // W, W^2, W^4, W^8
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

constexpr int kZBytes = kSl * kTcPoints * kTK * 2;  // one tile's Z' slices, as laid out in shared memory

struct TcSmem {
  uint16_t zq[kSl][kTK][kTcPoints];   // Z' slices (bf16 bits); rows kappa of the 64 points, chunks swizzled
  uint16_t aq[kSl][2 * kSub][kTK];    // A' slices of the current sub-tile
  xh w8[kTcPoints];                   // W^8 per point (64-bit mantissas)
  xh w1[kTcPoints];                   // W per point (the final combination)
  unsigned long long tm[kTB];         // tau^i = tm[i] 2^te[i]
  int te[kTB];
  int eq[kTcPoints];                  // Z' scale exponent per point
  int er[kSub];                       // A' scale exponent per block of the sub-tile
  int item, tile;
};

// Z' layout, per slice: 64 rows (kappa) of the 64 points' values (128 B), the
// 16-B chunk (8 points) xor-ed by kappa & 7; B fragments are read transposed
__device__ __forceinline__ int zswz(int kappa, int p) {
  return kappa * kTcPoints + ((((p >> 3) ^ (kappa & 7)) << 3) | (p & 7));
}

// a 128-bit value across lane ^ 1
__device__ __forceinline__ u128 shfl_u128_x1(u128 v) {
  const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, 1);
  const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), 1);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

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
// lies in [s_r + 64 q, s_r + 64 (q + 1)), so a group has about 64 points, or
// one bin with more.  A group's tilt, the union of its points' windows and
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
    const int ng = (s[q + 1] - s[q] + kTcPoints - 1) / kTcPoints;
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
  const int x0 = s[r] + kTcPoints * lg, x1 = x0 + kTcPoints;
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

// per tile point (one thread each): u = w / tau, the Z'
// slices of u^i (i < 32) written straight to global memory in the layout
// k_tc_sum copies into shared memory (for each slice and term, the 64
// points' values are one 128-B row, so a warp's stores are contiguous),
// W^(2^k) = (u^32 tau^32)^(2^k), and Z's scale exponent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcPoints) k_tc_pre(DevPoly P, const PointRec *__restrict__ rec,
                                                      const TcTile *__restrict__ tiles, TcPoint *__restrict__ pts,
                                                      const TcTau *__restrict__ taus, uint16_t *__restrict__ zglob,
                                                      const uint32_t *cnt) {
  const int ntiles = (int)cnt[kCntTcTiles], p = threadIdx.x;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
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
      cur = xh_norm(1ull << 63, 0, 0, 0, 0);  // 1
    }
    // powers u^i in 64-bit mantissas: each product truncates at 2^-63, so u^31
    // is within 2^-58 of its value relative to itself.  Lane pairs (points
    // p even, p + 1) share the stores: the even lane writes both points' real
    // parts, the odd lane both imaginary parts, each as bf16 pairs.
    const int odd = p & 1, pb = p & ~1;
    uint32_t *zt = reinterpret_cast<uint32_t *>(zglob + (size_t)t * (kZBytes / 2));
    for (int i = 0; i < kTB; ++i) {
      if (i > 0 && valid) cur = xh_mul(cur, uh);
      // x 2^(e - 63) 2^(70 - (eQ + 1)) = x 2^-sr: fixed point below 2^69 (components <= 2^(eQ - 1))
      const int sr = eQ + 1 - 7 - (int)cur.e;
      const u128 fr = valid ? shift_to70((u128)cur.x, sr) : (u128)0;
      const u128 fi = valid ? shift_to70((u128)cur.y, sr) : (u128)0;
      const u128 mine = odd ? fi : fr, recv = shfl_u128_x1(odd ? fr : fi);
      const uint32_t nmine = (uint32_t)(odd ? cur.sy : cur.sx);
      const uint32_t nrecv = __shfl_xor_sync(0xffffffffu, (uint32_t)(odd ? cur.sx : cur.sy), 1);
      uint32_t xa[kSl], xb[kSl];  // point pb, point pb + 1
      bchunks70(odd ? recv : mine, xa);
      bchunks70(odd ? mine : recv, xb);
      const DigitSign sa = digit_sign(odd ? nrecv : nmine), sb = digit_sign(odd ? nmine : nrecv);
      const int c = zswz(odd ? kTB + i : i, pb) >> 1;
#pragma unroll
      for (int s = 0; s < kSl; ++s) zt[s * (kTK * kTcPoints / 2) + c] = bf16_pair(xa[s], sa, xb[s], sb);
    }
    TcPoint o;
    xint W = zero;
    if (valid) {  // W = u^32 tau^32 = w^32 from the 128-bit u: the block weights W^g and
      // (W^8)^tau of the Horner must not inherit the 64-bit powers' error
      xint u32 = u;
      for (int k = 0; k < 5; ++k) u32 = xint_sqr(u32);
      W = xint_mul(u32, taus[t].tau32);
    }
    o.W[0] = W;
    for (int k = 1; k < 4; ++k) o.W[k] = xint_sqr(o.W[k - 1]);
    o.eq = eQ + 1;  // Z' = F 2^(eq - 70)
    o.pad[0] = o.pad[1] = o.pad[2] = 0;
    pts[(size_t)t * kTcPoints + p] = o;
  }
}

// ---------------------------------------------------------------------------
// the window sums: persistent CTAs of 8 warps (two per SM) take work items (a
// tile and a run of at most `chunk` blocks) from a counter; each item's
// value per point, sum over its blocks m of C_m W^(m - first), goes to a slot
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 2)
    k_tc_sum(DevPoly P, const TcTile *__restrict__ tiles, const TcPoint *__restrict__ pts,
             const TcTau *__restrict__ taus, const uint4 *__restrict__ zglob, const int32_t *__restrict__ item_base,
             const int32_t *__restrict__ item_tile, uint32_t *cnt, xint *__restrict__ slots) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t nitems = *(volatile uint32_t *)&cnt[kCntTcItems];
  const long long chunk = (long long)*(volatile uint32_t *)&cnt[kCntTcChunk];
  const xint zero = xint_norm(0, 0, 0, 0, 0);
  while (true) {
    if (tid == 0) {
      const uint32_t it = atomicAdd(&cnt[kCntTcWork], 1u);
      S.item = (int)it;
      S.tile = it < nitems ? item_tile[it] : -1;
    }
    __syncthreads();
    const int item = S.item, t = S.tile;
    if (t < 0) break;
    const TcTile T = tiles[t];
    const int j = T.piece;
    const long long k0 = P.piece_k0[j], k1 = (long long)P.piece_k0[j + 1] - 1;
    const long long mb = T.mlo + (long long)(item - item_base[t]) * chunk;
    const long long me = min((long long)(T.mlo + T.nblk), mb + chunk);
    const TcPoint *tp = pts + (size_t)t * kTcPoints;

    // ---- setup: the tile's Z' slices, tau^i, W^8 and Z's scales into shared memory
    {
      const uint4 *src = zglob + (size_t)t * (kZBytes / 16);
      uint4 *dst = reinterpret_cast<uint4 *>(&S.zq[0][0][0]);
      for (int i = tid; i < kZBytes / 16; i += kTcThreads) dst[i] = src[i];
      if (tid < kTB) {
        S.tm[tid] = taus[t].tm[tid];
        S.te[tid] = taus[t].te[tid];
      }
      if (tid < kTcPoints) {
        const bool v = tid < T.count;
        S.w8[tid] = xh_from_xint(v ? tp[tid].W[3] : zero);
        S.eq[tid] = v ? tp[tid].eq : 1;
        S.w1[tid] = xh_from_xint(v ? tp[tid].W[0] : zero);
      }
    }
    __syncthreads();

    // ---- sub-tiles of 8 blocks, from the top down (Horner in W^8 per lane)
    const int g = lane >> 2, tq = lane & 3;
    const int p0 = 8 * wid + 2 * tq;
    xh H0 = xh_norm(0, 0, 0, 0, 0), H1 = H0;
    const int nsub = (int)((me - mb + kSub - 1) / kSub);
    // coefficient of this lane in block mb + 8 ts + wid (0 outside the item or the piece)
    auto load_b = [&](int ts_) -> double2 {
      const long long m = mb + (long long)kSub * ts_ + wid;
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
    for (int ts = nsub - 1; ts >= 0; --ts) {
      const long long m0 = mb + (long long)kSub * ts;
      {  // A' for block m0 + wid, lane = term i
        const double br = bnext.x, bi = bnext.y;
        bnext = load_b(ts - 1);  // in flight during this sub-tile's MMAs
        const unsigned long long tmi = S.tm[lane];
        const int tei = S.te[lane];
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
        const u128 fr = pr ? shift_to70(pr, eR - 70 - er_) : (u128)0;
        const u128 fi = pi ? shift_to70(pi, eR - 70 - ei_) : (u128)0;
        const uint32_t nr = br < 0.0, ni = bi < 0.0;
        // lane pairs (terms i even, i + 1) share the stores: the even lane
        // takes both terms' real parts, the odd lane both imaginary parts
        const int odd = lane & 1, ib = lane & ~1;
        const u128 mine = odd ? fi : fr, recv = shfl_u128_x1(odd ? fr : fi);
        const uint32_t nmine = odd ? ni : nr, nrecv = __shfl_xor_sync(0xffffffffu, odd ? nr : ni, 1);
        uint32_t xa[kSl], xb[kSl];  // term ib, term ib + 1
        bchunks70(odd ? recv : mine, xa);
        bchunks70(odd ? mine : recv, xb);
        const DigitSign sa = digit_sign(odd ? nrecv : nmine), sb = digit_sign(odd ? nmine : nrecv);
        // out_re row (wid): ( A'_re | -A'_im ), out_im row (8 + wid): ( A'_im | A'_re ).
        // Even lane: the A'_re pair at (re row, low half) and (im row, high
        // half); odd lane: -A'_im at (re row, high half), A'_im at (im row, low half).
        const int c_lo = ((ib >> 3) ^ wid) << 3 | (ib & 7), c_hi = ((4 + (ib >> 3)) ^ wid) << 3 | (ib & 7);
        const int o_re = (wid * kTK + (odd ? c_hi : c_lo)) >> 1;
        const int o_im = ((kSub + wid) * kTK + (odd ? c_lo : c_hi)) >> 1;
        const uint32_t flip = odd ? 0x80008000u : 0u;
        uint32_t *a32 = reinterpret_cast<uint32_t *>(&S.aq[0][0][0]);
#pragma unroll
        for (int s = 0; s < kSl; ++s) {
          const uint32_t w = bf16_pair(xa[s], sa, xb[s], sb);
          a32[s * (kSub * kTK) + o_re] = w ^ flip;
          a32[s * (kSub * kTK) + o_im] = w;
        }
        if (lane == 0) S.er[wid] = eR;
      }
      __syncthreads();
      float acc[kSl][4];
#pragma unroll
      for (int s = 0; s < kSl; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = 0.0f;
#pragma unroll
      for (int kp = 0; kp < 2; ++kp) {
        uint32_t bq[kSl][4];
        {  // rows kappa = 32 kp + lane (8 per matrix), the warp's 8 points
          const int row = 32 * kp + lane;
#pragma unroll
          for (int s = 0; s < kSl; ++s)
            ldsm_x4_t(bq[s], &S.zq[s][0][0] + row * kTcPoints + ((wid ^ (row & 7)) << 3));
        }
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const int ks = 2 * kp + kk;
          const int row = (lane & 7) + 8 * ((lane >> 3) & 1), ch = 2 * ks + (lane >> 4);
#pragma unroll
          for (int sa = 0; sa < kSl; ++sa) {
            uint32_t a[4];
            ldsm_x4(a, &S.aq[sa][0][0] + row * kTK + ((ch ^ (row & 7)) << 3));
#pragma unroll
            for (int sz = 0; sz < kSl - sa; ++sz) mma_bf16(acc[sa + sz], a, bq[sz][2 * kk], bq[sz][2 * kk + 1]);
          }
        }
      }
      __syncthreads();  // the A' tile is free for the next sub-tile
      // combine: lane holds block m0 + g at points p0, p0 + 1
      const bool inblk = m0 + g < me;
      const int eRg = S.er[g];
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {
        const int p = p0 + pp;
        xh C = xh_norm(0, 0, 0, 0, 0);
        if (inblk && p < T.count) {
          u128 xr, xi;
          int sr, si;
          join_acc(acc, pp, xr, sr);
          join_acc(acc, 2 + pp, xi, si);
          C = xh_from128(xr, sr, xi, si, 49 + (long long)eRg + S.eq[p]);
        }
        xh &H = pp ? H1 : H0;
        if (H.x || H.y) H = xh_mul(H, S.w8[p]);
        H = xh_add(H, C);
      }
    }
    // ---- V = sum_g W^g H_g: the lanes' H into shared memory (over the Z'
    // tiles, no longer read), then one thread per point, Horner over g in
    // 64-bit mantissas (seven steps: within 2^-57 of the terms' sum)
    xh *hs = reinterpret_cast<xh *>(&S.zq[0][0][0]);  // [point][g]
    hs[p0 * kSub + g] = H0;
    hs[(p0 + 1) * kSub + g] = H1;
    __syncthreads();
    if (tid < T.count) {
      const xh W = S.w1[tid];
      xh V = hs[tid * kSub + kSub - 1];
      for (int gg = kSub - 2; gg >= 0; --gg) {
        if (V.x || V.y) V = xh_mul(V, W);
        V = xh_add(V, hs[tid * kSub + gg]);
      }
      slots[(size_t)item * kTcPoints + tid] = xint_from_xh(V);
    }
    __syncthreads();  // shared memory is reused by the next item
  }
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
// longer ones eight (L = 8): threads q < 7 take a contiguous seventh of the
// items by Horner in W^chunk and scale it by (W^chunk)^(its first item),
// thread 7 computes z^(kb + v) meanwhile, and the parts are added by
// shuffles.  Each launch skips the other's tiles.
constexpr int kFinOneLaneItems = 4;
template <int L>
__global__ void __launch_bounds__(L * kTcPoints)
    k_tc_finalize(DevPoly P, const PointRec *__restrict__ rec, const TcTile *__restrict__ tiles,
                  const TcPoint *__restrict__ pts, const int32_t *__restrict__ item_base, const uint32_t *cnt,
                  const xint *__restrict__ slots, fpe_xc64 *__restrict__ out, int32_t *nterms,
                  int32_t *bits_lost) {
  const int ntiles = (int)cnt[kCntTcTiles], p = threadIdx.x / L, q = threadIdx.x % L;
  constexpr int qpow = L - 1;            // the thread that computes z^(kb + v)
  constexpr int nh = L > 1 ? L - 1 : 1;  // threads that take items
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
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

static int64_t tc_groups_max(int64_t n) { return (n + kTcPoints - 1) / kTcPoints + kTcMaxPieces; }
static int64_t tc_tiles_max(int64_t n) { return (n + kTcPoints - 1) / kTcPoints + tc_groups_max(n); }
static int64_t tc_items_cap(int64_t n) { return tc_tiles_max(n) + (int64_t)tc_num_sms() * kTcItemsPerSm; }
constexpr int kTcCtasPerSm = 2;

bool tc_enabled(const fpe_poly_s *P, bool complex_points) {
  (void)complex_points;
  return P->dev.n_tc > 0 && !P->dev.fp32 && !P->dev.accurate && P->tune.tc_min_window > 0;
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
    cudaError_t e = cudaFuncSetAttribute(k_tc_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
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
    k_tc_pre<<<std::min(tm, tc_num_sms() * 16), kTcPoints, 0, st>>>(P->dev, w.rec, (const TcTile *)w.tc_tiles,
                                                                    (TcPoint *)w.tc_points,
                                                                    (const TcTau *)w.tc_taus, (uint16_t *)w.tc_z, cnt);
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
    k_tc_sum<<<tc_num_sms() * kTcCtasPerSm, kTcThreads, sizeof(TcSmem), st>>>(
        P->dev, (const TcTile *)w.tc_tiles, (const TcPoint *)w.tc_points, (const TcTau *)w.tc_taus,
        (const uint4 *)w.tc_z, w.tc_item_base, w.tc_item_tile, cnt, (xint *)w.tc_slots);
  }
  {
    ProfScope ps("k_tc_finalize", st, 2);  // eight- and one-thread launches
    k_tc_finalize<8><<<std::min(tm, tc_num_sms() * 2), 8 * kTcPoints, 0, st>>>(
        P->dev, w.rec, (const TcTile *)w.tc_tiles, (const TcPoint *)w.tc_points, w.tc_item_base, cnt,
        (const xint *)w.tc_slots, out, nterms, bits_lost);
    k_tc_finalize<1><<<std::min(tm, tc_num_sms() * 16), kTcPoints, 0, st>>>(
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
