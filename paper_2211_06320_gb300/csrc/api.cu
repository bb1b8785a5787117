// extern "C" entry points of fpe.h: argument checks, handle management,
// host-buffer staging, and kernel timing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fpe_internal.h"

namespace fpe {
const char *last_error_cstr();

// ------------------------------------------------------------------ timing
namespace {
struct ProfRec {
  std::string name;
  cudaEvent_t e0, e1;
  int kernels;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
}  // namespace

ProfScope::ProfScope(const char *n, cudaStream_t s, int k) : name(n), st(s), kernels(k) {
  if (!g_prof_on) return;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
}
ProfScope::~ProfScope() {
  if (!e0) return;
  cudaEventRecord(e1, st);
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof.push_back({name, e0, e1, kernels});
}

static fpe_status check_eval_args(fpe_poly_t P, const double *z_re, int64_t n, const void *out) {
  if (!P) {
    set_error("NULL handle");
    return FPE_ERR_INVALID_ARG;
  }
  if (P->flags & FPE_HOST_ONLY) {
    set_error("handle was preconditioned with FPE_HOST_ONLY");
    return FPE_ERR_INVALID_ARG;
  }
  if (n < 0 || n >= ((int64_t)1 << 31)) {
    set_error("n must be in [0, 2^31)");
    return FPE_ERR_INVALID_ARG;
  }
  if (n > 0 && (!z_re || !out)) {
    set_error("NULL point or output pointer");
    return FPE_ERR_INVALID_ARG;
  }
  return FPE_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace fpe

using namespace fpe;

// ---------------------------------------------------------------------------
// launch parameters and the autotuner
// ---------------------------------------------------------------------------

static fpe_status check_tuning(const fpe_tuning *t) {
  if (!t || t->long_window < 32 || t->long_window > (1 << 24) || t->lane_chunk < 16 || t->lane_chunk > (1 << 16)) {
    set_error("tuning: need long_window in [32, 2^24] and lane_chunk in [16, 2^16]");
    return FPE_ERR_INVALID_ARG;
  }
  return FPE_OK;
}

// Time run() at every setting of the grid, keep the fastest in tune.
template <class Run>
static fpe_status autotune_grid(Tuning &tune, double &tune_ms, Run run, cudaStream_t st, fpe_tuning *best) {
  static const int64_t kLW[] = {1024, 2048, 4096, 8192};
  static const int64_t kLC[] = {128, 256, 512, 1024, 2048};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  const Tuning keep = tune;
  Tuning pick = keep;
  double pick_ms = -1.0;
  fpe_status s = FPE_OK;
  for (int64_t lw : kLW) {
    for (int64_t lc : kLC) {
      tune.long_window = lw;
      tune.lane_chunk = lc;
      if ((s = run()) != FPE_OK) break;  // untimed
      if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
      if ((s = run()) != FPE_OK || (s = run()) != FPE_OK) break;
      if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (pick_ms < 0.0 || ms / 2.0 < pick_ms) {
        pick_ms = ms / 2.0;
        pick = tune;
      }
    }
    if (s != FPE_OK || e != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == FPE_OK && e != cudaSuccess) s = cuda_fail(e, "fpe_autotune timing");
  if (s != FPE_OK) {
    tune = keep;
    return s;
  }
  tune = pick;
  tune_ms = pick_ms;
  best->long_window = pick.long_window;
  best->lane_chunk = pick.lane_chunk;
  best->ms = pick_ms;
  return FPE_OK;
}

extern "C" {

fpe_status fpe_precondition(const double *re, const double *im, const int64_t *e2, int64_t n_coef, int p,
                            uint32_t flags, fpe_poly_t *out) {
  return precondition_host(re, im, e2, n_coef, p, flags, out);
}

fpe_status fpe_eval(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                    int32_t *nterms, int32_t *bits_lost, void *cuda_stream) {
  fpe_status s = check_eval_args(P, z_re, n, out);
  if (s != FPE_OK) return s;
  DeviceGuard g(P->device);
  return launch_eval(P, z_re, z_im, n, out, nterms, bits_lost, (cudaStream_t)cuda_stream);
}

fpe_status fpe_eval_host(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                         int32_t *nterms, int32_t *bits_lost) {
  fpe_status s = check_eval_args(P, z_re, n, out);
  if (s != FPE_OK) return s;
  if (n == 0) return FPE_OK;
  DeviceGuard g(P->device);
  // device staging: z (1 or 2 arrays), out, nterms, bits_lost
  const size_t nz = (z_im ? 2 : 1) * n * sizeof(double);
  const size_t no = n * sizeof(fpe_xc64), ni = n * sizeof(int32_t);
  const size_t need = nz + no + 2 * ni + 256;
  Workspace &w = P->ws;
  cudaError_t e;
  if (w.dev_io_bytes < need) {
    if (w.dev_io) cudaFree(w.dev_io);
    w.dev_io = nullptr;
    w.dev_io_bytes = 0;
    if ((e = cudaMalloc(&w.dev_io, need)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(io)");
    w.dev_io_bytes = need;
  }
  char *base = (char *)w.dev_io;
  double *dzr = (double *)base;
  double *dzi = z_im ? dzr + n : nullptr;
  fpe_xc64 *dout = (fpe_xc64 *)(base + nz);
  int32_t *dnt = nterms ? (int32_t *)(base + nz + no) : nullptr;
  int32_t *dbl = bits_lost ? (int32_t *)(base + nz + no + ni) : nullptr;
  cudaStream_t st = nullptr;
  if ((e = cudaMemcpyAsync(dzr, z_re, n * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(z)");
  if (z_im && (e = cudaMemcpyAsync(dzi, z_im, n * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(z)");
  s = launch_eval(P, dzr, dzi, n, dout, dnt, dbl, st);
  if (s != FPE_OK) return s;
  if ((e = cudaMemcpyAsync(out, dout, no, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(out)");
  if (nterms && (e = cudaMemcpyAsync(nterms, dnt, ni, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(nterms)");
  if (bits_lost && (e = cudaMemcpyAsync(bits_lost, dbl, ni, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(bits_lost)");
  return fpe_sync(P, st);
}

fpe_status fpe_eval_deriv(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                          void *cuda_stream) {
  fpe_status s = check_eval_args(P, z_re, n, out);
  if (s != FPE_OK) return s;
  if (!(P->flags & FPE_WITH_DERIV)) {
    set_error("fpe_eval_deriv: handle was preconditioned without FPE_WITH_DERIV");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  if (P->deriv_zero || !P->deriv) {
    cudaError_t e = cudaMemsetAsync(out, 0, n * sizeof(fpe_xc64), (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? FPE_OK : cuda_fail(e, "cudaMemsetAsync");
  }
  return launch_eval(P->deriv, z_re, z_im, n, out, nullptr, nullptr, (cudaStream_t)cuda_stream);
}

fpe_status fpe_batch_create(const fpe_poly_t *P, int64_t npoly, const int64_t *pt_offsets, fpe_batch_t *out) {
  if (!out) {
    set_error("fpe_batch_create: out is NULL");
    return FPE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!P || npoly < 1 || npoly > ((int64_t)1 << 26) || !pt_offsets || pt_offsets[0] != 0) {
    set_error("fpe_batch_create: need npoly >= 1 handles and offsets starting at 0");
    return FPE_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < npoly; ++i) {
    if (!P[i] || (P[i]->flags & FPE_HOST_ONLY) || pt_offsets[i + 1] < pt_offsets[i]) {
      set_error("fpe_batch_create: NULL or host-only handle, or decreasing offsets");
      return FPE_ERR_INVALID_ARG;
    }
    if (P[i]->device != P[0]->device || P[i]->complex_coef != P[0]->complex_coef ||
        P[i]->dev.fp32 != P[0]->dev.fp32 || P[i]->dev.accurate != P[0]->dev.accurate) {
      set_error("fpe_batch_create: all handles must share the device, real/complex coefficients, FPE_FP32 and "
                "FPE_ACCURATE");
      return FPE_ERR_UNSUPPORTED;
    }
  }
  const int64_t ntotal = pt_offsets[npoly];
  if (ntotal >= ((int64_t)1 << 31)) {
    set_error("fpe_batch_create: at most 2^31 - 1 points in a batch");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P[0]->device);
  fpe_batch_s *B = new fpe_batch_s();
  B->device = P[0]->device;
  B->npoly = npoly;
  B->ntotal = ntotal;
  B->complex_coef = P[0]->complex_coef;
  B->fp32 = P[0]->dev.fp32 != 0;
  B->accurate = P[0]->dev.accurate != 0;
  B->polys.assign(P, P + npoly);
  B->offsets.assign(pt_offsets, pt_offsets + npoly + 1);
  std::vector<DevPoly> table(npoly);
  for (int64_t i = 0; i < npoly; ++i) table[i] = P[i]->dev;
  std::vector<int32_t> pid(std::max<int64_t>(ntotal, 1));
  for (int64_t i = 0; i < npoly; ++i)
    for (int64_t j = pt_offsets[i]; j < pt_offsets[i + 1]; ++j) pid[j] = (int32_t)i;
  const int kBins = kBatchBins;
  cudaError_t e = cudaSuccess;
  auto A = [&e](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void **)&B->d_table, npoly * sizeof(DevPoly));
  A((void **)&B->d_pid, pid.size() * sizeof(int32_t));
  A((void **)&B->d_offsets, (npoly + 1) * sizeof(int64_t));
  A((void **)&B->d_hist, npoly * kBins * sizeof(uint32_t));
  A((void **)&B->d_cursor, npoly * kBins * sizeof(uint32_t));
  A((void **)&B->d_cnt, kNumCounters * sizeof(uint32_t));
  A((void **)&B->d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(B->d_table, table.data(), npoly * sizeof(DevPoly), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B->d_pid, pid.data(), pid.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(B->d_offsets, pt_offsets, (npoly + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(B->d_status, 0, sizeof(int32_t));
  fpe_status st = e == cudaSuccess ? alloc_workspace(B->ws, ntotal) : cuda_fail(e, "fpe_batch_create");
  if (st != FPE_OK) {
    fpe_batch_destroy(B);
    return st;
  }
  *out = B;
  return FPE_OK;
}

fpe_status fpe_batch_eval(fpe_batch_t B, const double *z_re, const double *z_im, fpe_xc64 *out, int32_t *nterms,
                          void *cuda_stream) {
  if (!B || (B->ntotal > 0 && (!z_re || !out))) {
    set_error("fpe_batch_eval: NULL batch, point or output pointer");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(B->device);
  return launch_batch(B, z_re, z_im, out, nterms, (cudaStream_t)cuda_stream);
}

fpe_status fpe_batch_sync(fpe_batch_t B, void *cuda_stream) {
  if (!B) {
    set_error("NULL batch");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(B->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int32_t h = 0;
  if ((e = cudaMemcpy(&h, B->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy(status)");
  if (h) {
    cudaMemset(B->d_status, 0, sizeof(int32_t));
    set_error("non-finite evaluation point");
    return FPE_ERR_NONFINITE;
  }
  return FPE_OK;
}

void fpe_batch_destroy(fpe_batch_t B) {
  if (!B) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(B->device);
  void *ptrs[] = {B->d_table, B->d_pid, B->d_offsets, B->d_hist, B->d_cursor, B->d_cnt, B->d_status};
  for (void *a : ptrs)
    if (a) cudaFree(a);
  free_workspace(B->ws);
  if (prev >= 0) cudaSetDevice(prev);
  delete B;
}

fpe_status fpe_set_tuning(fpe_poly_t P, const fpe_tuning *t) {
  if (!P) {
    set_error("fpe_set_tuning: NULL handle");
    return FPE_ERR_INVALID_ARG;
  }
  fpe_status s = check_tuning(t);
  if (s != FPE_OK) return s;
  P->tune.long_window = t->long_window;
  P->tune.lane_chunk = t->lane_chunk;
  P->tune_ms = 0.0;
  return FPE_OK;
}

fpe_status fpe_get_tuning(fpe_poly_t P, fpe_tuning *t) {
  if (!P || !t) {
    set_error("fpe_get_tuning: NULL handle or output");
    return FPE_ERR_INVALID_ARG;
  }
  t->long_window = P->tune.long_window;
  t->lane_chunk = P->tune.lane_chunk;
  t->ms = P->tune_ms;
  return FPE_OK;
}

fpe_status fpe_set_tensor_path(fpe_poly_t P, int64_t min_window) {
  if (!P || (min_window != 0 && (min_window < 32 || min_window > ((int64_t)1 << 30)))) {
    set_error("fpe_set_tensor_path: NULL handle, or min_window not 0 and outside [32, 2^30]");
    return FPE_ERR_INVALID_ARG;
  }
  P->tune.tc_min_window = min_window;
  P->tune.tc_min_points = 0;  // an explicit setting applies to calls of every size
  return FPE_OK;
}

fpe_status fpe_get_tensor_path(fpe_poly_t P, int64_t *min_window, int32_t *n_pieces) {
  if (!P) {
    set_error("fpe_get_tensor_path: NULL handle");
    return FPE_ERR_INVALID_ARG;
  }
  if (min_window) *min_window = P->tune.tc_min_window;
  if (n_pieces) *n_pieces = P->dev.n_tc;
  return FPE_OK;
}

fpe_status fpe_autotune(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, void *cuda_stream,
                        fpe_tuning *best) {
  fpe_tuning dummy;
  fpe_status s = check_eval_args(P, z_re, n, &dummy);
  if (s != FPE_OK) return s;
  if (!best || n == 0) {
    set_error("fpe_autotune: need best != NULL and n > 0");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  fpe_xc64 *out = nullptr;
  cudaError_t e = cudaMalloc((void **)&out, n * sizeof(fpe_xc64));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(autotune)");
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  s = autotune_grid(P->tune, P->tune_ms,
                    [&]() { return launch_eval(P, z_re, z_im, n, out, nullptr, nullptr, st); }, st, best);
  cudaStreamSynchronize(st);
  cudaFree(out);
  return s;
}

fpe_status fpe_batch_set_tuning(fpe_batch_t B, const fpe_tuning *t) {
  if (!B) {
    set_error("fpe_batch_set_tuning: NULL batch");
    return FPE_ERR_INVALID_ARG;
  }
  fpe_status s = check_tuning(t);
  if (s != FPE_OK) return s;
  B->tune.long_window = t->long_window;
  B->tune.lane_chunk = t->lane_chunk;
  return FPE_OK;
}

fpe_status fpe_batch_autotune(fpe_batch_t B, const double *z_re, const double *z_im, void *cuda_stream,
                              fpe_tuning *best) {
  if (!B || !best || B->ntotal == 0 || !z_re) {
    set_error("fpe_batch_autotune: NULL batch, points or output, or an empty batch");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(B->device);
  fpe_xc64 *out = nullptr;
  cudaError_t e = cudaMalloc((void **)&out, B->ntotal * sizeof(fpe_xc64));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(autotune)");
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  double ms = 0.0;
  fpe_status s = autotune_grid(B->tune, ms, [&]() { return launch_batch(B, z_re, z_im, out, nullptr, st); }, st,
                               best);
  cudaStreamSynchronize(st);
  cudaFree(out);
  return s;
}

fpe_status fpe_eval_batch(const fpe_poly_t *P, int64_t npoly, const int64_t *pt_offsets, const double *z_re,
                          const double *z_im, fpe_xc64 *out, void *cuda_stream) {
  if (npoly == 0) return FPE_OK;
  fpe_batch_t B = nullptr;
  fpe_status s = fpe_batch_create(P, npoly, pt_offsets, &B);
  if (s != FPE_OK) return s;
  s = fpe_batch_eval(B, z_re, z_im, out, nullptr, cuda_stream);
  if (s == FPE_OK) s = fpe_batch_sync(B, cuda_stream);
  fpe_batch_destroy(B);
  return s;
}

fpe_status fpe_newton(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *inc,
                      double *z_next_re, double *z_next_im, void *cuda_stream) {
  fpe_status s = check_eval_args(P, z_re, n, inc);
  if (s != FPE_OK) return s;
  if (!(P->flags & FPE_WITH_DERIV)) {
    set_error("fpe_newton: handle was preconditioned without FPE_WITH_DERIV");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  return launch_newton(P, z_re, z_im, n, inc, z_next_re, z_next_im, (cudaStream_t)cuda_stream);
}

fpe_status fpe_grad_points(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, const double *g_re,
                           const double *g_im, double *gz_re, double *gz_im, void *cuda_stream) {
  fpe_status s = check_eval_args(P, z_re, n, gz_re);
  if (s != FPE_OK) return s;
  if (!(P->flags & FPE_WITH_DERIV) || (n > 0 && !g_re)) {
    set_error("fpe_grad_points: needs FPE_WITH_DERIV and a non-NULL g_re");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  return launch_grad_points(P, z_re, z_im, n, g_re, g_im, gz_re, gz_im, (cudaStream_t)cuda_stream);
}

fpe_status fpe_grad_coeffs(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, const double *g_re,
                           const double *g_im, double *ga_re, double *ga_im, void *cuda_stream) {
  fpe_status s = check_eval_args(P, z_re, n, ga_re);
  if (s != FPE_OK) return s;
  if (n > 0 && !g_re) {
    set_error("fpe_grad_coeffs: g_re is NULL");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  return launch_grad_coeffs(P, z_re, z_im, n, g_re, g_im, ga_re, ga_im, (cudaStream_t)cuda_stream);
}

fpe_status fpe_to_complex(const fpe_xc64 *v, int64_t n, double *re, double *im, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!v || !re))) {
    set_error("fpe_to_complex: bad arguments");
    return FPE_ERR_INVALID_ARG;
  }
  return launch_to_complex(v, n, re, im, (cudaStream_t)cuda_stream);
}

fpe_status fpe_horner(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                      int compensated, void *cuda_stream) {
  fpe_status s = check_eval_args(P, z_re, n, out);
  if (s != FPE_OK) return s;
  DeviceGuard g(P->device);
  return launch_horner(P, z_re, z_im, n, out, compensated, (cudaStream_t)cuda_stream);
}

fpe_status fpe_info(fpe_poly_t P, int64_t *d, int64_t *valuation, int64_t *n_hull, int64_t *n_good, int *T) {
  if (!P) {
    set_error("NULL handle");
    return FPE_ERR_INVALID_ARG;
  }
  if (d) *d = P->d;
  if (valuation) *valuation = P->v;
  if (n_hull) *n_hull = (int64_t)P->hull_k.size();
  if (n_good) *n_good = P->n_good;
  if (T) *T = P->T;
  return FPE_OK;
}

fpe_status fpe_get_hull(fpe_poly_t P, int64_t *k, int64_t *s, int64_t cap) {
  if (!P || !k || !s || cap < (int64_t)P->hull_k.size()) {
    set_error("fpe_get_hull: bad arguments or capacity too small");
    return FPE_ERR_INVALID_ARG;
  }
  std::memcpy(k, P->hull_k.data(), P->hull_k.size() * sizeof(int64_t));
  std::memcpy(s, P->hull_s.data(), P->hull_s.size() * sizeof(int64_t));
  return FPE_OK;
}

fpe_status fpe_get_good(fpe_poly_t P, uint8_t *mask, int64_t n_coef) {
  if (!P || !mask || n_coef != P->n_coef) {
    set_error("fpe_get_good: bad arguments");
    return FPE_ERR_INVALID_ARG;
  }
  std::memcpy(mask, P->good.data(), (size_t)n_coef);
  return FPE_OK;
}

fpe_status fpe_get_windows(fpe_poly_t P, int64_t n, int64_t *l, int64_t *r, double *N, void *cuda_stream) {
  if (!P || (P->flags & FPE_HOST_ONLY) || n != P->last_n || n > P->ws.cap) {
    set_error("fpe_get_windows: n must equal the size of the last fpe_eval");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSuccess;
  if (l && e == cudaSuccess) e = cudaMemcpyAsync(l, P->ws.lo, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  if (r && e == cudaSuccess) e = cudaMemcpyAsync(r, P->ws.hi, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  if (N && e == cudaSuccess) e = cudaMemcpyAsync(N, P->ws.N, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? FPE_OK : cuda_fail(e, "cudaMemcpyAsync");
}

fpe_status fpe_analyse(fpe_poly_t P, double *lam_lo, double *lam_hi, int64_t n_coef) {
  if (!P || !lam_lo || !lam_hi || n_coef != P->n_coef) {
    set_error("fpe_analyse: bad arguments");
    return FPE_ERR_INVALID_ARG;
  }
  const std::vector<int64_t> &hk = P->hull_k, &hs = P->hull_s;
  const int nh = (int)hk.size();
  const double T = (double)P->T;
  const double nan = std::nan("");
  // cover(k) + lambda k >= max_i (s_i + lambda k_i) - T  <=>  for every vertex i:
  //   lambda (k - k_i) >= s_i - cover(k) - T
  for (int64_t k = 0; k < n_coef; ++k) {
    if (!P->good[k]) {
      lam_lo[k] = lam_hi[k] = nan;
      continue;
    }
    // cover(k) exactly as a rational on its segment, evaluated in FP64
    int seg = 0;
    while (seg + 1 < nh - 1 && hk[seg + 1] <= k) ++seg;
    double cov = (double)hs[seg];
    if (nh > 1 && k != hk[seg])
      cov = (double)hs[seg] + (double)(hs[seg + 1] - hs[seg]) * (double)(k - hk[seg]) / (double)(hk[seg + 1] - hk[seg]);
    double lo = -INFINITY, hi = INFINITY;
    for (int i = 0; i < nh; ++i) {
      if (hk[i] < k) lo = fmax(lo, ((double)hs[i] - cov - T) / (double)(k - hk[i]));
      else if (hk[i] > k) hi = fmin(hi, (cov + T - (double)hs[i]) / (double)(hk[i] - k));
    }
    lam_lo[k] = lo;
    lam_hi[k] = hi;
  }
  return FPE_OK;
}

fpe_status fpe_sync(fpe_poly_t P, void *cuda_stream) {
  if (!P || (P->flags & FPE_HOST_ONLY)) {
    set_error("NULL handle");
    return FPE_ERR_INVALID_ARG;
  }
  DeviceGuard g(P->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int32_t h = 0;
  if ((e = cudaMemcpy(&h, P->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy(status)");
  if (h) {
    cudaMemset(P->d_status, 0, sizeof(int32_t));
    if (h & kStatusNonFinite) {
      set_error("non-finite evaluation point");
      return FPE_ERR_NONFINITE;
    }
    if (h & kStatusTimeout) {
      set_error("a bounded wait of the tensor-core window sums gave up (results are incomplete)");
      return FPE_ERR_TIMEOUT;
    }
    set_error("device status " + std::to_string(h));
    return FPE_ERR_CUDA;
  }
  return FPE_OK;
}

void fpe_destroy(fpe_poly_t P) { free_handle(P); }

const char *fpe_status_string(fpe_status s) {
  switch (s) {
    case FPE_OK: return "ok";
    case FPE_ERR_INVALID_ARG: return "invalid argument";
    case FPE_ERR_NONFINITE: return "non-finite input";
    case FPE_ERR_ZERO_POLY: return "zero polynomial";
    case FPE_ERR_OOM: return "out of memory";
    case FPE_ERR_CUDA: return "CUDA error";
    case FPE_ERR_TIMEOUT: return "device wait timed out";
    case FPE_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *fpe_last_error(void) { return last_error_cstr(); }

void fpe_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof_on = on != 0;
}

void fpe_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto &r : g_prof) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  g_prof.clear();
}

fpe_status fpe_profile_read(const char *name, double *total_ms, int64_t *launches) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  double tot = 0.0;
  int64_t cnt = 0;
  for (auto &r : g_prof) {
    if (name && !std::strstr(r.name.c_str(), name)) continue;
    cudaError_t e = cudaEventSynchronize(r.e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    tot += ms;
    cnt += r.kernels;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = cnt;
  return FPE_OK;
}

}  // extern "C"
