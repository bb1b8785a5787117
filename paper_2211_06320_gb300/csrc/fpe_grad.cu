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
//                    depends on no other coefficient.
//   fpe_to_complex   (re, im) 2^e as plain FP64 (inf where it overflows).
#include <cuda_runtime.h>

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

// One thread per point (bucketed order): walks the point's window upward,
// c_k = g conj(z)^k kept as an FP64 mantissa pair and an exponent,
// renormalised every 32 steps; adds c_k to dL/da_k for every good k.
template <bool CZ>
__global__ void __launch_bounds__(128) k_grad_coeffs(DevPoly P, int n, const PointRec *__restrict__ rec,
                                                     const double *__restrict__ gre,
                                                     const double *__restrict__ gim, double *__restrict__ gar,
                                                     double *__restrict__ gai) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const PointRec r = rec[q];
  const double gr = gre[r.orig], gi = gim ? gim[r.orig] : 0.0;
  if (r.flags) {
    // z = 0: P(0) = a_0, so only a_0 moves it (when a_0 is a coefficient of the valuation-0 part)
    if ((r.flags & kPointZero) && P.v == 0) {
      atomicAdd(&gar[0], gr);
      if (gai) atomicAdd(&gai[0], gi);
    }
    return;
  }
  const double cz_r = r.zr, cz_i = CZ ? -r.zi : 0.0;  // conj(z)
  // c = g conj(z)^(v + lo) in extended form
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
    if (((t - r.lo) & 31) == 31) {
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

fpe_status launch_newton(fpe_poly_s *P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *inc,
                         double *znr, double *zni, cudaStream_t st) {
  if (n == 0) return FPE_OK;
  void *buf = nullptr;
  fpe_status s = aux_buffer(P, 2 * n * sizeof(fpe_xc64), &buf);
  if (s != FPE_OK) return s;
  fpe_xc64 *Pv = (fpe_xc64 *)buf, *Dv = Pv + n;
  if ((s = launch_eval(P, z_re, z_im, n, Pv, nullptr, nullptr, st)) != FPE_OK) return s;
  if ((s = eval_deriv_into(P, z_re, z_im, n, Dv, st)) != FPE_OK) return s;
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
  {
    ProfScope ps("k_grad_coeffs", st);
    if (z_im)
      k_grad_coeffs<true><<<(int)((n + 127) / 128), 128, 0, st>>>(P->dev, (int)n, P->ws.rec, g_re, g_im, ga_re,
                                                                  ga_im);
    else
      k_grad_coeffs<false><<<(int)((n + 127) / 128), 128, 0, st>>>(P->dev, (int)n, P->ws.rec, g_re, g_im, ga_re,
                                                                   ga_im);
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
