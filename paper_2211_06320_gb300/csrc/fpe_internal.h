// Internal declarations shared by the host preconditioner (precondition.cpp),
// the CUDA kernels (fpe_eval.cu, fpe_horner.cu) and the ABI glue (api.cu).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <limits>
#include <string>
#include <vector>

#include "fpe.h"

namespace fpe {

// Coefficient "pieces": the trimmed index range [0, D] is cut at every
// multiple of the piece length (128 in FP64, 32 in FP32) and at every cover
// vertex.  On piece j the coefficients are stored as b_k = a_k * 2^-rho(k) with
// rho(k) = rho0[j] + beta[j] * (k - k0[j]) an integer line that follows the
// cover to within half a piece length plus one bit, so that every kept b_k
// lies in [2^-(T + len/2 + 3), 2^(len/2 + 2)] and Horner's recurrence on piece
// j runs at the exactly rescaled point w_j = 2^beta[j] * z.
constexpr int kLog2PieceLen = 7;       // FP64 coefficients
constexpr int kLog2PieceLenF32 = 5;    // FP32 coefficients: keeps b_k and partial sums inside FP32 range

// Packed integer copy of the FPE coefficients, read by the integer-pipe
// window sums: each component (-1)^s m 2^e (m < 2^53) is a 54-bit
// two's-complement mantissa in bits 0..53 and e + kQBias in bits 54..63, so
// the device gets (mantissa, exponent) with two shifts.  Kept coefficients
// have e in [-(T + 67) - 52, 14] (the bounds above), well inside the field;
// a component with e < -kQBias (below 2^-459, negligible beside the other
// component of a kept coefficient) or a zero is stored as 0.
constexpr int kQBias = 512;

// Scale of the FP32 rounding-error bookkeeping of the FP64 window sums:
// magnitudes are kept as |x| 2^kMagOff (fpe_device.cuh, fpe_window.cuh).
constexpr int kMagOff = 60;

// A lower bound of |br + i bi| 2^kMagOff as a float: the FP64 modulus with a
// margin above its rounding (two squares, a sum and a root err by under
// 3 2^-53), rounded down to FP32; 0 below the FP32 range, the largest float
// above it.  One per kept coefficient (DevPoly::bmag).
inline float coef_mag_lo(double br, double bi) {
  const double a = std::sqrt(br * br + bi * bi) * (1.0 - 0x1p-50);
  const double x = std::ldexp(a, kMagOff);
  if (!(x > 0.0)) return 0.0f;
  if (x >= (double)std::numeric_limits<float>::max()) return std::numeric_limits<float>::max();
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, 0.0f);
  return f;
}

// the packed word of x, or ~0 when x's exponent does not fit the field
inline uint64_t qpack(double x) {
  if (x == 0.0) return 0;
  int ex;
  const double f = std::frexp(x, &ex);  // x = f 2^ex, 0.5 <= |f| < 1
  const long long m = (long long)std::ldexp(f, 53);  // exact
  const int e = ex - 53;
  if (e < -kQBias) return 0;
  if (e >= kQBias) return ~(uint64_t)0;
  return ((uint64_t)(e + kQBias) << 54) | ((uint64_t)m & ((1ull << 54) - 1));
}

// Resident 128-thread blocks per SM asked of the window-sum kernels (caps
// their registers at 65536 / (128 * this)); the persistent ones
// (k_sum_groups, k_sums) are launched with exactly this many blocks per SM.
#ifndef FPE_SUM_BLOCKS_PER_SM
#define FPE_SUM_BLOCKS_PER_SM 4
#endif
constexpr int kSumBlocksPerSm = FPE_SUM_BLOCKS_PER_SM;

// Threads per block of k_sum_short when the tensor-core sums run beside it:
// three warps (12288 registers) fit on an SM beside one k_tc_sum CTA
// (17 warps of 96 registers), so the FP64 pipe keeps working while the
// tensor and integer pipes take the long windows.
#ifndef FPE_SHORT_THREADS_TC
#define FPE_SHORT_THREADS_TC 96
#endif
constexpr int kShortThreadsTc = FPE_SHORT_THREADS_TC;
static_assert(kShortThreadsTc % 32 == 0 && kShortThreadsTc <= 128, "whole warps, within the launch bound");

// How fpe_eval runs the tensor-core sums against the FP64 ones: 0 one after
// the other on the caller's stream; 1 on a second stream of the handle with
// the highest priority, forked from and joined back into the caller's
// stream; 2 the same at the default priority.
#ifndef FPE_TC_CONCURRENT
#define FPE_TC_CONCURRENT 1
#endif

// Bucketing of points by log2|z| before summation (points of similar modulus
// get similar windows; §8.1 suggests grouping evaluations of similar size).
constexpr int kNumBins = 4096;

// Points whose window is longer than the long-window threshold are summed
// by warp groups: a group is 32 lane chunks of at most lane_chunk terms, and
// a window gets ceil(L / (32 lane_chunk)) groups, so no warp's serial chain
// exceeds lane_chunk terms however long the window is; shorter windows get
// one thread each (32 points per warp).  Both are per-handle launch
// parameters (fpe_set_tuning, fpe_autotune); these are the defaults.
constexpr int64_t kLongWindow = 4096;
constexpr int64_t kMaxLaneChunk = 1024;
struct Tuning {
  int64_t long_window = kLongWindow;
  int64_t lane_chunk = kMaxLaneChunk;
  int64_t tc_min_window = 384;  // tensor-core window sums for windows of at least this many terms (0: off)
  int64_t tc_min_points = 32768;  // ... on calls of at least this many points (0 once set explicitly)
  int64_t group_span() const { return 32 * lane_chunk; }
};

// Tensor-core window sums (fpe_tc.cu).  Windows of at least tc_min_window
// terms that lie inside one long merged piece (an integer cover slope) are
// summed as exact integer products of 7-bit digits on the bf16 tensor cores.
// Their points are bucketed separately: kTcBinsPerPiece bins per such piece
// (at most kTcMaxPieces per polynomial), on a logarithmic scale of
// mu = log2|z| + beta, so consecutive points have nearly equal windows.
constexpr int kTcMaxPieces = 4;
constexpr int kTcBinsPerPiece = 32768;
constexpr int kTcBinsPerBinade = 512;  // over |mu| in [2^-24, 2^8], negative mu first
static_assert(32 * kTcBinsPerBinade <= kTcBinsPerPiece / 2, "32 binades of |mu| on each side of 0");
constexpr int kTcBins = kTcMaxPieces * kTcBinsPerPiece;
constexpr int kTcMinPieceLen = 64;  // shorter pieces never get the tensor path
constexpr int kTcPoints = 128;      // points per tile: the M = 128 rows of one tcgen05 MMA
constexpr int kTcItemsPerSm = 16;   // work items per SM the planner aims at (at least)
constexpr int kTcMinChunk = 256;    // blocks (of 32 terms) per work item, at least

// Batched evaluation: lambda bins per polynomial (segmented bucketing).
constexpr int kBatchBins = 32;

// Counters after the 2 * kNumBins histogram words.
constexpr int kCntLong = 0;        // long-window points listed
constexpr int kCntGroupWork = 1;   // group work cursor
constexpr int kCntExtra = 2;       // extra group slots reserved (groups 1.. of very long windows)
constexpr int kCntFinal = 3;       // finalize cursor
constexpr int kCntTcStart = 4;     // 5 words: bucketed start of each tensor-core piece's points, then n
constexpr int kCntTcWork = 9;      // tensor-core work cursor
constexpr int kCntTcItems = 10;    // tensor-core work items
constexpr int kCntTcChunk = 11;    // blocks per tensor-core work item
constexpr int kCntTcTiles = 12;    // tensor-core tiles
constexpr int kCntTcSubtiles = 13; // tensor-core MMA sub-tiles
constexpr int kCntTcPoints = 14;   // points summed on the tensor cores
constexpr int kCntTcRejected = 15; // tensor-core points handed back to the FP64 kernels
constexpr int kCntResum = 16;      // short windows whose FP64 sum was not certified, listed for the exact re-sum
constexpr int kNumCounters = 17;

// Device view of a preconditioned polynomial, passed to kernels by value.
struct DevPoly {
  const double *b;             // FPE coefficients (bad ones zeroed), trimmed k = 0..D;
                               // complex: interleaved (re, im); real: one double
  const double *b_full;        // every coefficient, same layout (Horner baselines)
  const float *bf;             // FPE_FP32: the FPE coefficients rounded to FP32 (same layout)
  const uint64_t *bq;          // the FPE coefficients packed by qpack (same layout; FP64 modes)
  const float *bmag;           // FP64 modes: coef_mag_lo of each FPE coefficient, k = 0..D
  const int32_t *piece_k0;     // npieces + 1 entries, last = D + 1
  const int32_t *piece_beta;   // integer slope of rho on the piece
  const int32_t *piece_delta;  // exponent shift applied to h when entering piece j from j + 1
  const int64_t *piece_rho0;   // rho at the piece's first index
  const int32_t *piece_first;  // per block of 2^log2_piece indices: first piece overlapping it
  const double *hull_k;        // trimmed abscissae of the cover's vertices
  const double *hull_s;        // their scales
  const double *hull_sig;      // slopes of the n_hull - 1 segments
  const int32_t *gcount;       // gcount[k] = #{good j < k}, D + 2 entries
  const int32_t *good_idx;     // the good (trimmed) indices in increasing order, gcount[D + 1] entries
  int64_t D;                   // trimmed degree d - v
  int64_t v;                   // valuation (first nonzero index)
  double T;                    // p + s(d) + 3
  int32_t n_hull;
  int32_t npieces;
  int32_t complex_coef;
  int32_t fp32;
  int32_t accurate;    // FPE_ACCURATE: window sums on the integer pipe
  int32_t sparse_mode;  // 0: sparse window sums where G_p fills at most a quarter of the window; 1: never; 2: always
  int32_t log2_piece;  // kLog2PieceLen or kLog2PieceLenF32
  double a0_re, a0_im;  // a_0 as a normalised mantissa (0 when v > 0)
  int64_t a0_e;
  int32_t tc_piece[kTcMaxPieces];  // pieces eligible for the tensor-core window sums
  int32_t n_tc;                    // how many (0: none)
};

// One evaluation point after location, in bucketed order.
struct PointRec {
  double zr, zi;
  long long lo, hi;  // window in trimmed indices; lo > hi: no window (z = 0 or non-finite)
  long long kl;      // k_lambda (trimmed): the window's peak term
  double N;          // max of cover(k) + lambda k, untrimmed (eq. defN)
  int32_t orig;      // index in the caller's order
  int32_t flags;     // kPointZero, kPointNonFinite
  int32_t pid;       // polynomial of the point (batched evaluation; 0 otherwise)
  int32_t pad;
};
constexpr int32_t kPointZero = 1;
constexpr int32_t kPointNonFinite = 2;
constexpr int32_t kPointTC = 4;  // summed by the tensor-core kernels

// Device status word bits.
constexpr int32_t kStatusNonFinite = 1;
constexpr int32_t kStatusTimeout = 2;  // a bounded device-side wait gave up

// Scratch memory of one handle, grown on demand.
struct Workspace {
  int64_t cap = 0;
  long long *lo = nullptr, *hi = nullptr;  // per point, caller order (untrimmed)
  long long *kl = nullptr;                 // per point, caller order (trimmed k_lambda)
  double *N = nullptr;
  uint32_t *key = nullptr;       // per point, caller order: bucket key; at key + cap, its place in the bin
  PointRec *rec = nullptr;       // bucketed order
  int32_t *long_list = nullptr;     // bucketed positions of long-window points
  int32_t *long_ngroups = nullptr;  // warp groups per long-window point
  int32_t *long_gbase = nullptr;    // first extra group slot (groups 1..)
  int32_t *extra_owner = nullptr;   // per extra group slot: long-point index
  int32_t *extra_group = nullptr;   // per extra group slot: group number
  void *group_val = nullptr;        // per group: value (40-byte extended double-double)
  void *group_carry = nullptr;      // per group: carry into the next group
  int64_t extra_cap = 0;            // extra group slots (after the cap group-0 slots)
  uint32_t *bins = nullptr;         // 2 * nbins histogram words, kNumCounters counters, tile totals
  int nbins = kNumBins;             // bins of the last front pass (kNumBins, or + kTcBins with the tensor path)
  void *tc_tiles = nullptr;         // TcTile per tile
  int32_t *tc_item_base = nullptr;  // first work item of each tile (tiles + 1 entries)
  void *tc_slots = nullptr;         // per work item and tile point: the chunk's value (xint)
  void *tc_points = nullptr;        // TcPoint per tile point
  int32_t *tc_item_tile = nullptr;  // tile of each work item
  void *tc_taus = nullptr;          // TcTau per tile
  void *tc_z = nullptr;             // Z' slices per tile
  void *tc_groups = nullptr;        // TcGroup per group of bins
  void *tc_plan = nullptr;          // planning scratch (totals; per group tiles, first tile, first item)
  int64_t tc_cap = 0;               // points the tensor-core arrays are sized for
  void *host_pinned = nullptr;   // staging for fpe_eval_host
  size_t host_pinned_bytes = 0;
  void *dev_io = nullptr;        // device staging for fpe_eval_host
  size_t dev_io_bytes = 0;
};

}  // namespace fpe

struct fpe_poly_s {
  fpe::DevPoly dev{};
  int device = 0;
  int p = 53;
  uint32_t flags = 0;
  int64_t n_coef = 0, d = 0, v = 0;
  int T = 0;
  bool complex_coef = false;
  std::vector<int64_t> hull_k, hull_s;  // untrimmed
  std::vector<uint8_t> good;            // untrimmed mask, n_coef entries
  int64_t n_good = 0;
  std::vector<void *> allocs;           // device allocations owned by the handle
  fpe::Workspace ws;
  int32_t *d_status = nullptr;          // device status word
  fpe_poly_s *deriv = nullptr;          // P' (FPE_WITH_DERIV), nullptr if P' = 0
  bool deriv_zero = false;
  int64_t last_n = 0;                   // points of the last fpe_eval
  void *aux = nullptr;                  // scratch of fpe_newton / fpe_grad_points (grown on demand)
  size_t aux_bytes = 0;
  fpe::Tuning tune;                     // launch parameters of the window sums
  double tune_ms = 0.0;                 // time per call of the setting fpe_autotune chose
  cudaStream_t tc_stream = nullptr;     // the tensor-core sums' stream (created on first use)
  cudaEvent_t tc_fork = nullptr, tc_join = nullptr;  // its fork from and join into the caller's stream
};

struct fpe_batch_s {
  int device = 0;
  int64_t npoly = 0, ntotal = 0;
  bool complex_coef = false, fp32 = false, accurate = false;
  std::vector<fpe_poly_s *> polys;      // not owned
  std::vector<int64_t> offsets;         // npoly + 1 point offsets
  fpe::DevPoly *d_table = nullptr;      // npoly descriptors
  int32_t *d_pid = nullptr;             // per point: polynomial index
  int64_t *d_offsets = nullptr;
  uint32_t *d_hist = nullptr, *d_cursor = nullptr;  // npoly * kBatchBins each
  uint32_t *d_cnt = nullptr;            // kNumCounters
  int32_t *d_status = nullptr;
  fpe::Workspace ws;                    // sized for ntotal points
  fpe::Tuning tune;                     // launch parameters of the window sums
};

namespace fpe {
// precondition.cpp
fpe_status alloc_workspace(Workspace &w, int64_t n);
void free_workspace(Workspace &w);
fpe_status precondition_host(const double *re, const double *im, const int64_t *e2, int64_t n_coef, int p,
                             uint32_t flags, fpe_poly_s **out);
void set_error(const std::string &msg);
fpe_status cuda_fail(cudaError_t e, const char *what);
void free_handle(fpe_poly_s *P);
fpe_status ensure_workspace(fpe_poly_s *P, int64_t n);

// fpe_eval.cu
fpe_status launch_front(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, cudaStream_t st,
                        bool allow_tc = false);
fpe_status launch_eval(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                       int32_t *nterms, int32_t *bits_lost, cudaStream_t st);
fpe_status launch_batch(fpe_batch_s *B, const double *z_re, const double *z_im, fpe_xc64 *out, int32_t *nterms,
                        cudaStream_t st);
// fpe_tc.cu: the tensor-core window sums of the points launch_front marked kPointTC
// (tc_plan runs before the other window kernels: it hands back tiles it rejects)
bool tc_enabled(const fpe_poly_s *P, bool complex_points, int64_t n);
fpe_status ensure_tc_workspace(fpe_poly_s *P, int64_t n);
fpe_status launch_tc_groups(fpe_poly_s *P, int n, cudaStream_t st);
fpe_status launch_tc_plan(fpe_poly_s *P, int n, cudaStream_t st);
fpe_status launch_tc_sums(fpe_poly_s *P, int n, fpe_xc64 *out, int32_t *nterms, int32_t *bits_lost,
                          cudaStream_t st);
void free_tc_workspace(Workspace &w);
// fpe_grad.cu
fpe_status launch_newton(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *inc,
                         double *znr, double *zni, cudaStream_t st);
fpe_status launch_grad_points(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n,
                              const double *g_re, const double *g_im, double *gz_re, double *gz_im,
                              cudaStream_t st);
fpe_status launch_grad_coeffs(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n,
                              const double *g_re, const double *g_im, double *ga_re, double *ga_im,
                              cudaStream_t st);
fpe_status launch_to_complex(const fpe_xc64 *v, int64_t n, double *re, double *im, cudaStream_t st);
// fpe_horner.cu
fpe_status launch_horner(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                         int compensated, cudaStream_t st);

// kernel timing (api.cu)
struct ProfScope {  // events around `kernels` consecutive kernel launches on st
  const char *name;
  cudaStream_t st;
  int kernels;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(const char *name, cudaStream_t st, int kernels = 1);
  ~ProfScope();
};
}  // namespace fpe
