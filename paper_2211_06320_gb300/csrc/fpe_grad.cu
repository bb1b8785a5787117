// Newton step and derivatives on top of the evaluation path (§7.2).
//
//   fpe_newton       N_P(z) = z - P(z)/P'(z) (eq. newton).  P and P' come from
//                    the FPE path as extended-exponent values, so their ratio
//                    never overflows even where P(z) and P'(z) do: the
//                    exponents subtract, which is what the paper obtains by
//                    cancelling the valuation monomial z^m, m = min(l, l').
//   fpe_grad_points  dL/dz = g conj(P'(z)) for an upstream gradient g = dL/dP
//                    (conjugate Wirtinger convention: P is holomorphic in z).
//   fpe_grad_coeffs  dL/da_k += sum_j g_j conj(z_j)^k over the kept terms
//                    k in G_p cap [l_j, r_j] of each point: the FPE output
//                    depends on no other coefficient.  Short windows: a warp
//                    sums its 32 points per coefficient in shared memory
//                    before one atomic add; long windows: a warp per point,
//                    lanes on consecutive coefficients.
//   fpe_to_complex   (re, im) 2^e as plain FP64 (inf where it overflows).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <map>
#include <mutex>

#include "fpe_device.cuh"
#include "fpe_internal.h"

namespace fpe {

__global__ void k_newton_combine(int n, const fpe_xc64 *__restrict__ Pv, const fpe_xc64 *__restrict__ Dv,
                                 const double *__restrict__ zre, const double *__restrict__ zim,
                                 fpe_xc64 *__restrict__ inc, double *__restrict__ znr, double *__restrict__ zni) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const fpe_xc64 a = Pv[j], b = Dv[j];
  fpe_xc64 q;
  if (a.re == 0.0 && a.im == 0.0) {
    q.re = q.im = 0.0;  // at a root the increment is 0 (also when P' vanishes there)
    q.e = 0;
  } else if (b.re == 0.0 && b.im == 0.0) {
    q.re = q.im = __longlong_as_double(0x7ff8000000000000ll);  // P'(z) = 0, P(z) != 0: undefined
    q.e = 0;
  } else {
    // (a.re + i a.im) / (b.re + i b.im) with both mantissas in [0.5, 1): no overflow
    const double den = fma(b.re, b.re, b.im * b.im);
    const double qr = fma(a.re, b.re, a.im * b.im) / den;
    const double qi = fma(a.im, b.re, -a.re * b.im) / den;
    const int f = frexp_exp(fmax(fabs(qr), fabs(qi)));
    q.re = scale2(qr, -f);
    q.im = scale2(qi, -f);
    q.e = a.e - b.e + f;
  }
  inc[j] = q;
  if (znr) {
    const int ee = (int)max(-3000LL, min(3000LL, (long long)q.e));
    znr[j] = zre[j] - scale2(q.re, ee);
    if (zni) zni[j] = (zim ? zim[j] : 0.0) - scale2(q.im, ee);
  }
}

__global__ void k_grad_points(int n, const double *__restrict__ gre, const double *__restrict__ gim,
                              const fpe_xc64 *__restrict__ Dv, double *__restrict__ ozr, double *__restrict__ ozi) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const fpe_xc64 d = Dv[j];
  const int ee = (int)max(-3000LL, min(3000LL, (long long)d.e));
  const double dr = scale2(d.re, ee), di = scale2(d.im, ee);
  const double gr = gre[j], gi = gim ? gim[j] : 0.0;
  // g conj(P')
  ozr[j] = fma(gr, dr, gi * di);
  if (ozi) ozi[j] = fma(gi, dr, -gr * di);
}

// One thread walks one point's window upward: c_k = g conj(z)^k kept as an
// FP64 mantissa pair and an exponent, renormalised every 8 steps; adds c_k to
// dL/da_k for every good k.  Used for warps whose points are far apart in
// |z| (see k_grad_coeffs_short).
template <bool CZ>
__device__ __forceinline__ void grad_point_atomic(const DevPoly &P, const PointRec &r, double gr, double gi,
                                                  double *__restrict__ gar, double *__restrict__ gai) {
  const double cz_r = r.zr, cz_i = CZ ? -r.zi : 0.0;  // conj(z)
  xdd pw = xdd_pow_int(cz_r, cz_i, P.v + r.lo);
  xdd c = xdd_mul_d(pw, gr, gi, 0);
  double cr = c.rh + c.rl, ci = c.ih + c.il;
  long long ce = c.e;
  for (long long t = r.lo; t <= r.hi; ++t) {
    if (P.gcount[t + 1] != P.gcount[t]) {
      const int sh = (int)max(-3000LL, min(3000LL, ce));
      atomicAdd(&gar[P.v + t], scale2(cr, sh));
      if (gai) atomicAdd(&gai[P.v + t], scale2(ci, sh));
    }
    const double nr = fma(cr, cz_r, -ci * cz_i), ni = fma(cr, cz_i, ci * cz_r);
    cr = nr;
    ci = ni;
    if (((t - r.lo) & 7) == 7) {
      const double m = fmax(fabs(cr), fabs(ci));
      if (m != 0.0) {
        const int f = frexp_exp(m);
        cr = scale2(cr, -f);
        ci = scale2(ci, -f);
        ce += f;
      }
    }
  }
}

__device__ __forceinline__ double warp_max_d(double x) {
  for (int s = 16; s >= 1; s >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, s));
  return x;
}
__device__ __forceinline__ long long warp_max_ll(long long x) {
  for (int s = 16; s >= 1; s >>= 1) x = max(x, (long long)__shfl_xor_sync(0xffffffffu, x, s));
  return x;
}
__device__ __forceinline__ long long warp_min_ll(long long x) {
  for (int s = 16; s >= 1; s >>= 1) x = min(x, (long long)__shfl_xor_sync(0xffffffffu, x, s));
  return x;
}

// Short windows, 32 bucketed points per warp (one per lane).  The warp walks
// the union of its lanes' windows 8 coefficients at a time: each lane writes
// its contributions g conj(z)^k (0 outside its window) into a shared tile,
// then lane l < 16 sums row l (coefficient k0 + (l & 7), component l >> 3)
// over the 32 points and makes the one atomic add for it: one atomic per
// coefficient component per warp instead of one per point.  The lanes keep
// one exponent E, renormalised after every tile; a warp whose points' |z|
// differ too much for that (powers more than 2^400 apart over the union)
// takes the one-thread-per-point loop instead.
constexpr int kGradTile = 8;

template <bool CZ>
__global__ void __launch_bounds__(128) k_grad_coeffs_short(DevPoly P, int n, const PointRec *__restrict__ rec,
                                                           const double *__restrict__ gre,
                                                           const double *__restrict__ gim,
                                                           double *__restrict__ gar, double *__restrict__ gai,
                                                           long long long_window) {
  __shared__ double tile[4][2][kGradTile][33];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  PointRec r;
  bool act = false;
  double gr = 0.0, gi = 0.0;
  if (q < n) {
    r = rec[q];
    gr = gre[r.orig];
    gi = gim ? gim[r.orig] : 0.0;
    if (r.flags) {
      // z = 0: P(0) = a_0, so only a_0 moves it (when a_0 is a coefficient of the valuation-0 part)
      if ((r.flags & kPointZero) && P.v == 0) {
        atomicAdd(&gar[0], gr);
        if (gai) atomicAdd(&gai[0], gi);
      }
    } else {
      act = r.hi - r.lo + 1 <= long_window;
    }
  }
  const long long ulo = warp_min_ll(act ? r.lo : LLONG_MAX), uhi = warp_max_ll(act ? r.hi : LLONG_MIN);
  if (ulo > uhi) return;  // no short window in this warp (warp-uniform)
  // spread of |z| over the warp, in bits over the union window
  const double lam = act ? log2(fmax(fabs(r.zr), fabs(r.zi))) : 0.0;
  const double lmax = warp_max_d(act ? lam : -1e300), lmin = -warp_max_d(act ? -lam : -1e300);
  if ((lmax - lmin) * (double)(uhi - ulo + 1) > 400.0) {
    if (act) grad_point_atomic<CZ>(P, r, gr, gi, gar, gai);
    return;
  }
  const double cz_r = act ? r.zr : 0.0, cz_i = (act && CZ) ? -r.zi : 0.0;  // conj(z)
  double cr = 0.0, ci = 0.0;
  long long ce = LLONG_MIN / 2;
  if (act) {
    const xdd c = xdd_mul_d(xdd_pow_int(cz_r, cz_i, P.v + ulo), gr, gi, 0);
    cr = c.rh + c.rl;
    ci = c.ih + c.il;
    if (cr != 0.0 || ci != 0.0) ce = c.e;
  }
  long long E = warp_max_ll(ce);
  if (E == LLONG_MIN / 2) return;  // every g is 0 (warp-uniform)
  {
    const int sh = (int)max(-3000LL, ce - E);  // <= 0
    cr = scale2(cr, sh);
    ci = scale2(ci, sh);
  }
  for (long long k0 = ulo; k0 <= uhi; k0 += kGradTile) {
#pragma unroll
    for (int kk = 0; kk < kGradTile; ++kk) {
      const long long k = k0 + kk;
      const bool in = act && k >= r.lo && k <= r.hi;
      tile[wib][0][kk][lane] = in ? cr : 0.0;
      tile[wib][1][kk][lane] = in ? ci : 0.0;
      const double nr = fma(cr, cz_r, -ci * cz_i), ni = fma(cr, cz_i, ci * cz_r);
      cr = nr;
      ci = ni;
    }
    __syncwarp();
    if (lane < 2 * kGradTile) {
      const int kk = lane & (kGradTile - 1), comp = lane / kGradTile;
      const long long k = k0 + kk;
      if (k <= uhi && P.gcount[k + 1] != P.gcount[k] && (comp == 0 || gai)) {
        double sum = 0.0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) sum += tile[wib][comp][kk][j];
        if (sum != 0.0) atomicAdd(&(comp ? gai : gar)[P.v + k], scale2(sum, (int)max(-3000LL, min(3000LL, E))));
      }
    }
    __syncwarp();
    const double m = warp_max_d(fmax(fabs(cr), fabs(ci)));
    if (m != 0.0 && isfinite(m)) {
      const int f = frexp_exp(m);
      cr = scale2(cr, -f);
      ci = scale2(ci, -f);
      E += f;
    }
  }
}

// Long windows, one warp per point: lane i takes k = l + i + 32 m, so the
// 32 atomic adds of a step go to 32 different coefficients.  Each lane starts
// from g conj(z)^(v + l + i) and multiplies by conj(z)^32 held in
// double-double (8 FMA per step), with its own exponent renormalised every 8
// steps; the drift is that of L/32 FP64 roundings.
template <bool CZ>
__global__ void __launch_bounds__(128) k_grad_coeffs_long(DevPoly P, const PointRec *__restrict__ rec,
                                                          const int32_t *__restrict__ long_list,
                                                          const uint32_t *cnt, const double *__restrict__ gre,
                                                          const double *__restrict__ gim,
                                                          double *__restrict__ gar, double *__restrict__ gai) {
  const int lane = threadIdx.x & 31;
  const uint32_t nlong = *(volatile const uint32_t *)&cnt[kCntLong];
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nlong; i += nwarps) {
    const PointRec r = rec[long_list[i]];
    const double gr = gre[r.orig], gi = gim ? gim[r.orig] : 0.0;
    const double cz_r = r.zr, cz_i = CZ ? -r.zi : 0.0;  // conj(z)
    const xdd c0 = xdd_mul_d(xdd_pow_int(cz_r, cz_i, P.v + r.lo + lane), gr, gi, 0);
    double cr = c0.rh + c0.rl, ci = c0.ih + c0.il;
    long long ce = c0.e;
    const xdd M = xdd_pow_int(cz_r, cz_i, 32);  // conj(z)^32 = (mh + ml) 2^me
    const double mhr = M.rh, mlr = M.rl, mhi = M.ih, mli = M.il;
    const long long me = M.e;
    int steps = 0;
    for (long long k = r.lo + lane; k <= r.hi; k += 32) {
      if (P.gcount[k + 1] != P.gcount[k]) {
        const int sh = (int)max(-3000LL, min(3000LL, ce));
        atomicAdd(&gar[P.v + k], scale2(cr, sh));
        if (gai) atomicAdd(&gai[P.v + k], scale2(ci, sh));
      }
      double nr, ni;
      if (CZ) {
        nr = fma(cr, mhr, fma(-ci, mhi, fma(cr, mlr, -ci * mli)));
        ni = fma(cr, mhi, fma(ci, mhr, fma(cr, mli, ci * mlr)));
      } else {
        nr = fma(cr, mhr, cr * mlr);
        ni = fma(ci, mhr, ci * mlr);
      }
      cr = nr;
      ci = ni;
      ce += me;
      if (++steps == 8) {
        steps = 0;
        const double m = fmax(fabs(cr), fabs(ci));
        if (m != 0.0 && isfinite(m)) {
          const int f = frexp_exp(m);
          cr = scale2(cr, -f);
          ci = scale2(ci, -f);
          ce += f;
        }
      }
    }
  }
}

__global__ void k_to_complex(int n, const fpe_xc64 *__restrict__ v, double *__restrict__ re,
                             double *__restrict__ im) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const fpe_xc64 x = v[j];
  const int ee = (int)max(-3000LL, min(3000LL, (long long)x.e));
  re[j] = scale2(x.re, ee);
  if (im) im[j] = scale2(x.im, ee);
}

static fpe_status aux_buffer(fpe_poly_s *P, size_t bytes, void **out) {
  if (P->aux_bytes < bytes) {
    if (P->aux) cudaFree(P->aux);
    P->aux = nullptr;
    P->aux_bytes = 0;
    cudaError_t e = cudaMalloc(&P->aux, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(aux)");
    P->aux_bytes = bytes;
  }
  *out = P->aux;
  return FPE_OK;
}

// P'(z) into D (zero when P' = 0)
static fpe_status eval_deriv_into(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *D,
                                  cudaStream_t st) {
  if (P->deriv_zero || !P->deriv) {
    cudaError_t e = cudaMemsetAsync(D, 0, n * sizeof(fpe_xc64), st);
    return e == cudaSuccess ? FPE_OK : cuda_fail(e, "cudaMemsetAsync");
  }
  return launch_eval(P->deriv, z_re, z_im, n, D, nullptr, nullptr, st);
}

// fpe_newton evaluates P' on a second stream while P runs on the caller's
// stream: the two evaluations use separate handles (workspaces, status words,
// tensor-core streams) and separate halves of the scratch, so they can share
// the GPU, and each fills the other's serial stretches (the fronts, the
// planning launches, the exact re-sums).  One such stream per device, with
// its fork and join events, is created on first use and kept until exit; the
// mutex makes each fork / launch / join sequence atomic against other host
// threads, which share the stream and the events.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static std::mutex g_side_mu;
static std::map<int, SideStream> g_side;  // by device; guarded by g_side_mu

static fpe_status side_stream(int device, SideStream **out) {
  SideStream &ss = g_side[device];
  cudaError_t e = cudaSuccess;
  if (!ss.s && (e = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  if (!ss.fork && (e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreateWithFlags");
  if (!ss.join && (e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreateWithFlags");
  *out = &ss;
  return FPE_OK;
}

fpe_status launch_newton(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *inc,
                         double *znr, double *zni, cudaStream_t st) {
  if (n == 0) return FPE_OK;
  void *buf = nullptr;
  fpe_status s = aux_buffer(P, 2 * n * sizeof(fpe_xc64), &buf);
  if (s != FPE_OK) return s;
  fpe_xc64 *Pv = (fpe_xc64 *)buf, *Dv = Pv + n;
  if (P->deriv_zero || !P->deriv) {
    if ((s = launch_eval(P, z_re, z_im, n, Pv, nullptr, nullptr, st)) != FPE_OK) return s;
    if ((s = eval_deriv_into(P, z_re, z_im, n, Dv, st)) != FPE_OK) return s;
  } else {
    std::lock_guard<std::mutex> lk(g_side_mu);
    SideStream *ss = nullptr;
    if ((s = side_stream(P->device, &ss)) != FPE_OK) return s;
    cudaError_t e = cudaEventRecord(ss->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->s, ss->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "Newton stream fork");
    const fpe_status sp = launch_eval(P, z_re, z_im, n, Pv, nullptr, nullptr, st);
    const fpe_status sd = launch_eval(P->deriv, z_re, z_im, n, Dv, nullptr, nullptr, ss->s);
    e = cudaEventRecord(ss->join, ss->s);  // join, also after a failed launch
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ss->join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "Newton stream join");
    if (sp != FPE_OK) return sp;
    if (sd != FPE_OK) return sd;
  }
  {
    ProfScope ps("k_newton_combine", st);
    k_newton_combine<<<(int)((n + 255) / 256), 256, 0, st>>>((int)n, Pv, Dv, z_re, z_im, inc, znr, zni);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "k_newton_combine");
}

fpe_status launch_grad_points(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n,
                              const double *g_re, const double *g_im, double *gz_re, double *gz_im,
                              cudaStream_t st) {
  if (n == 0) return FPE_OK;
  void *buf = nullptr;
  fpe_status s = aux_buffer(P, n * sizeof(fpe_xc64), &buf);
  if (s != FPE_OK) return s;
  fpe_xc64 *Dv = (fpe_xc64 *)buf;
  if ((s = eval_deriv_into(P, z_re, z_im, n, Dv, st)) != FPE_OK) return s;
  {
    ProfScope ps("k_grad_points", st);
    k_grad_points<<<(int)((n + 255) / 256), 256, 0, st>>>((int)n, g_re, g_im, Dv, gz_re, gz_im);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "k_grad_points");
}

fpe_status launch_grad_coeffs(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n,
                              const double *g_re, const double *g_im, double *ga_re, double *ga_im,
                              cudaStream_t st) {
  if (n == 0) return FPE_OK;
  fpe_status s = launch_front(P, z_re, z_im, n, st);
  if (s != FPE_OK) return s;
  Workspace &w = P->ws;
  {
    ProfScope ps("k_grad_coeffs_short", st);
    if (z_im)
      k_grad_coeffs_short<true><<<(int)((n + 127) / 128), 128, 0, st>>>(P->dev, (int)n, w.rec, g_re, g_im, ga_re,
                                                                        ga_im, P->tune.long_window);
    else
      k_grad_coeffs_short<false><<<(int)((n + 127) / 128), 128, 0, st>>>(P->dev, (int)n, w.rec, g_re, g_im, ga_re,
                                                                         ga_im, P->tune.long_window);
  }
  {
    ProfScope ps("k_grad_coeffs_long", st);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(sms, 1) * 8;
    if (z_im)
      k_grad_coeffs_long<true><<<blocks, 128, 0, st>>>(P->dev, w.rec, w.long_list, w.bins + 2 * w.nbins, g_re, g_im,
                                                       ga_re, ga_im);
    else
      k_grad_coeffs_long<false><<<blocks, 128, 0, st>>>(P->dev, w.rec, w.long_list, w.bins + 2 * w.nbins, g_re,
                                                        g_im, ga_re, ga_im);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "k_grad_coeffs");
}

fpe_status launch_to_complex(const fpe_xc64 *v, int64_t n, double *re, double *im, cudaStream_t st) {
  if (n == 0) return FPE_OK;
  k_to_complex<<<(int)((n + 255) / 256), 256, 0, st>>>((int)n, v, re, im);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "k_to_complex");
}

}  // namespace fpe
