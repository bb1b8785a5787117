/*
 * fpe.h -- C ABI of a GPU (sm_103a) implementation of the fast polynomial
 * evaluator of Anton, Mihalache and Vigneron, "Fast Evaluation of Real and
 * Complex Polynomials" (arXiv 2211.06320).
 *
 * Problem (Alg. A_p, §4.3): given coefficients a_0..a_d and a precision p,
 * precondition once (scales s(a_k), concave cover of k -> s(a_k), good index
 * set G_p), then evaluate at many points z the reduced polynomial
 *     Q_lambda(z) = sum_{k in G_p cap [l, r]} a_k z^k          (eq. reducedQlambda)
 * where lambda = log2|z| and [l, r] is the largest integer interval on which
 * the cover plus lambda*k stays within T = p + s(d) + 3 of its maximum N
 * (def. LRN).  Thm. equivAlgo: Q_lambda(z) is as accurate as Horner over all
 * terms.
 *
 * Conventions for every call:
 *  - Errors are returned, never thrown; nothing is written to outputs on an
 *    argument error.  Device-side conditions (non-finite points) are recorded
 *    in the handle and returned by fpe_sync().
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device (e.g. torch tensor data); "host" pointers are ordinary memory.
 *  - The caller owns every buffer it passes; a handle owns its own device
 *    copies and its scratch memory, freed by fpe_destroy().
 *  - Calls on one handle must not run concurrently from several host threads,
 *    and evaluations on one handle must not overlap on different streams
 *    (they share the handle's scratch memory).  fpe_destroy() must not race
 *    with work in flight on the handle.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream); the
 *    evaluation calls are asynchronous on it unless stated otherwise.
 */
#ifndef FPE_H_
#define FPE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque preconditioned polynomial (host metadata plus device arrays). */
typedef struct fpe_poly_s *fpe_poly_t;

/* Extended-exponent complex value (re + i*im) * 2^e.  Normalised:
 * max(|re|, |im|) lies in [0.5, 1), or re = im = 0 and e = 0.  24 bytes. */
typedef struct {
  double re, im;
  int64_t e;
} fpe_xc64;

typedef enum {
  FPE_OK = 0,
  FPE_ERR_INVALID_ARG = 1, /* NULL handle/pointer, negative size, bad p or flags  */
  FPE_ERR_NONFINITE = 2,   /* a coefficient or an evaluation point is NaN or inf  */
  FPE_ERR_ZERO_POLY = 3,   /* every coefficient is zero                           */
  FPE_ERR_OOM = 4,         /* host or device allocation failed                    */
  FPE_ERR_CUDA = 5,        /* a CUDA runtime call failed (see fpe_last_error)     */
  FPE_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up                  */
  FPE_ERR_UNSUPPORTED = 7  /* valid request this build does not implement         */
} fpe_status;

/* fpe_precondition flags */
enum {
  FPE_REAL = 1,        /* treat the coefficients as real (im ignored)           */
  FPE_WITH_DERIV = 2,  /* also precondition P' for fpe_eval_deriv               */
  FPE_FP32 = 4,        /* FP32 mode (requires p <= 24): coefficients rounded to
                          FP32 and windows summed on the FP32 pipe with a
                          float-float multiplier; the window search and the
                          exponent bookkeeping stay FP64/integer.  Error
                          <= 2^-21 sum |a_k||z|^k for p = 24 (same caveat on
                          aligned terms as the default FP64 summation).
                          Not combinable with FPE_ACCURATE.                    */
  FPE_HOST_ONLY = 8,   /* host analysis only (scales, cover, G_p; the -analyse
                          task of §8.1): no device memory is touched and the
                          handle cannot be evaluated                           */
  FPE_ACCURATE = 16,   /* window sums on the integer pipe in 128-bit fixed
                          point: error <= u|P| + (2^-84 + L 2^-100) S for
                          every input (L = window length), at ~1.7x the time
                          of the default summation (see fpe_eval)              */
  FPE_FORCE_DENSE = 32,  /* never use the sparse window sums (see fpe_eval)  */
  FPE_FORCE_SPARSE = 64  /* use the sparse window sums for every window of
                            the FP64 modes (see fpe_eval); not combinable
                            with FPE_FORCE_DENSE                             */
};

/*
 * fpe_precondition -- preconditioning of Alg. A_p (§5.1).
 *
 * Computes the exact integer scales s(a_k) = 1 + floor(log2|a_k|) (eq. dsz),
 * the concave cover of k -> s(a_k) over the nonzero coefficients (def. EP),
 * the offset T = p + s(d) + 3 and the good set G_p = {k : s(a_k) >= cover(k)
 * - T} (eq. threshold), then uploads the coefficients to the current device
 * with bad ones zeroed.
 *
 *   re, im   host arrays of n_coef doubles: a_k = (re[k] + i*im[k]) * 2^e2[k].
 *            im == NULL (or flag FPE_REAL) gives a real polynomial.
 *   e2       host array of n_coef int64 binary exponents, or NULL for all 0;
 *            lets coefficients exceed the FP64 range.  |e2[k]| < 2^40.
 *   n_coef   d + 1 >= 1 (leading zeros are trimmed: d is the last nonzero
 *            index, v the first; z^v is factored out as in §4.3).
 *   p        precision in significand bits, 2 <= p <= 53 (p <= 24 with FPE_FP32).
 *   flags    FPE_REAL | FPE_WITH_DERIV | FPE_FP32 | FPE_HOST_ONLY | FPE_ACCURATE,
 *            FPE_FORCE_DENSE or FPE_FORCE_SPARSE.
 *   out      receives the handle.
 * Synchronous (uploads finish before return).  Errors: FPE_ERR_INVALID_ARG,
 * FPE_ERR_NONFINITE (a coefficient is NaN/inf), FPE_ERR_ZERO_POLY, FPE_ERR_OOM,
 * FPE_ERR_CUDA.
 */
fpe_status fpe_precondition(const double *re, const double *im, const int64_t *e2, int64_t n_coef, int p,
                            uint32_t flags, fpe_poly_t *out);

/*
 * fpe_eval -- evaluation of Alg. A_p (§5.2) at n points.
 *
 * For each point: lambda = log2|z| (eq. defLambda), k_lambda = argmax of
 * cover(k) + lambda*k by binary search on the cover's slopes (eq. defN),
 * [l, r] by two binary searches (def. LRN), and
 *     out[j] = z^l * sum_{k in G_p cap [l, r]} a_k z^{k-l}
 * summed by Horner over the window (eq. complexityAlgo) with exact
 * power-of-two rescaling, so no intermediate overflows.  z = 0 gives a_0.
 *
 *   z_re, z_im  device arrays of n doubles; z_im == NULL means real points.
 *   n           number of points, 0 <= n < 2^31.
 *   out         device array of n fpe_xc64 (the value of P(z_j)).
 *   nterms      device int32[n] or NULL: #(G_p cap [l, r]) per point.
 *   bits_lost   device int32[n] or NULL: estimated leading bits cancelled,
 *               max(0, ceil(N) - e) (Remark rmk:cancel, eq. slice).
 * Summation: by default each window up to the long-window length (see
 * fpe_set_tuning) is summed in FP64 toward its peak term (top-down above
 * k_lambda, bottom-up with a double-double 1/z below), and
 * every such sum carries a rounding-error certificate: beside the value the
 * loop keeps, in FP32 rounded outward, a rigorous bound E of its rounding
 * errors (half an ulp of each rounded result, carried by |w|) and a lower
 * bound S' of its term magnitudes.  A window whose E plus the output
 * rounding exceeds 7.6 u S' is summed again exactly on the integer pipe (as
 * with FPE_ACCURATE), so for every input
 *     |P_gpu - P| <= 2^-50 sum |a_k||z|^k   (FP64 modes, p = 53),
 * with the dropped terms of §6 inside that budget (fpe_cert_stats counts the
 * re-summed windows).  Longer windows are cut into lane chunks that are
 * summed exactly on the integer pipe, as with FPE_ACCURATE, and so is every
 * window of real points with real coefficients (on this GPU that costs less
 * than FP64 with certificates).  Windows of at least 384 terms inside one coefficient
 * piece are summed exactly on the tensor cores (fpe_set_tensor_path).  A
 * window with at most a quarter of its indices in G_p (FPE_FORCE_SPARSE: any
 * window; FPE_FORCE_DENSE: none) is summed over its good indices alone, by
 * Horner's scheme with power jumps z^(k' - k) in 128-bit fixed point on the
 * integer pipe (error below L 2^-119 S, no certificate needed).
 * With FPE_ACCURATE the window is summed top-down by Horner's scheme on
 * the integer pipe: the partial sum is a complex 128-bit fixed-point value
 * with a 64-bit exponent, the point is used exactly, and each step truncates
 * at 2^-104 or less of the partial sum, so the error is at most
 * u|P| + (2^-84 + L 2^-100) S for every input (u|P| from rounding the
 * output to FP64, 2^-84 S from the power z^l).
 * Asynchronous on cuda_stream.  The first call (and any call with a larger n
 * than before) allocates scratch memory on the handle.  When the tensor-core
 * sums run, the call forks them onto a second stream of the handle (created
 * on the first such call, at the device's highest stream priority) through
 * an event recorded on cuda_stream, and makes cuda_stream wait for them
 * through a second event: work queued on cuda_stream after the call sees
 * every output.  A handle's calls must not overlap on the GPU
 * (the handle's scratch is shared), so one handle is driven from one stream
 * at a time.  Non-finite points give NaN outputs and FPE_ERR_NONFINITE from
 * the next fpe_sync().
 */
fpe_status fpe_eval(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                    int32_t *nterms, int32_t *bits_lost, void *cuda_stream);

/*
 * fpe_eval_noalloc -- fpe_eval for callers that cannot allocate device memory
 * while they evaluate (the paper has no counterpart: it is a property of this
 * library, not of the method).  Examples: a process whose device-memory budget
 * is fixed at start-up, a latency-bound loop that must not pay for cudaMalloc
 * and the device synchronisation it implies, a host program that gives the
 * library only the buffers it owns.  fpe_eval allocates its per-call scratch
 * on the handle; this call instead uses one built-in scratch array of
 * 9,429,248 bytes (about 9.0 MiB) in the library's device memory, which every GPU
 * that loads the library holds until the process exits.
 *
 *   Arguments and results as fpe_eval (device pointers, async on cuda_stream).
 *   n            0 <= n <= 32768 points; larger n returns FPE_ERR_INVALID_ARG
 *                with a message (use fpe_eval, or split the points).
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls, on every handle and stream, share the one array: calls that overlap
 * on the GPU race and give wrong results; serialise them (one stream, or
 * events).  The array keeps the last call's contents; each call clears what it
 * needs cleared (the bucket histogram) itself.
 */
fpe_status fpe_eval_noalloc(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                            int32_t *nterms, int32_t *bits_lost, void *cuda_stream);

/*
 * fpe_eval_host -- fpe_eval on host buffers: copies z to the device, evaluates,
 * copies the results back and waits for them.  Same arguments as fpe_eval
 * with host pointers (nterms, bits_lost may be NULL).  Synchronous; returns
 * the device-side status as fpe_sync() would.
 */
fpe_status fpe_eval_host(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                         int32_t *nterms, int32_t *bits_lost);

/*
 * fpe_eval_deriv -- P'(z) (§7.2: derivative coefficients j*a_j, rounded once
 * to the FP64 mantissa, preconditioned separately as the paper allows).
 * Requires FPE_WITH_DERIV at preconditioning, else FPE_ERR_INVALID_ARG.
 * Arguments as fpe_eval (device pointers).
 */
fpe_status fpe_eval_deriv(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                          void *cuda_stream);

/*
 * Batched evaluation -- many polynomials, each at its own points (§8.1: the
 * algorithm is embarrassingly parallel over points): three kernels locate,
 * bucket and scatter the points, then one persistent launch does every
 * window sum from a device work counter.
 *
 * fpe_batch_create builds a batch over npoly handles (all on one device, all
 * real or all complex, the same FPE_FP32 and FPE_ACCURATE flags; otherwise
 * FPE_ERR_UNSUPPORTED).  Polynomial i owns points pt_offsets[i] ..
 * pt_offsets[i+1]-1 (HOST array of npoly+1 nondecreasing int64 starting at 0,
 * total below 2^31).  It uploads the polynomials' descriptors and allocates
 * the scratch for every point once; the handles must outlive the batch and
 * must not be re-preconditioned.  Synchronous.
 *
 * fpe_batch_eval evaluates all points: z_re, z_im (z_im NULL = real points)
 * are device arrays of pt_offsets[npoly] doubles, out a device array of that
 * many fpe_xc64, nterms a device int32 array or NULL.  It allocates nothing
 * and does not synchronise, so the call can be recorded into a CUDA graph on
 * a capturing stream and replayed.  Calls on one batch must not overlap.
 *
 * fpe_batch_sync waits for cuda_stream and returns FPE_ERR_NONFINITE if a
 * point was NaN/inf since the last sync.  fpe_batch_destroy frees the batch.
 *
 * fpe_eval_batch is the one-shot form: create, evaluate, sync, destroy
 * (synchronous; use the batch handle to evaluate the same polynomials again).
 */
typedef struct fpe_batch_s *fpe_batch_t;
fpe_status fpe_batch_create(const fpe_poly_t *P, int64_t npoly, const int64_t *pt_offsets, fpe_batch_t *out);
fpe_status fpe_batch_eval(fpe_batch_t B, const double *z_re, const double *z_im, fpe_xc64 *out, int32_t *nterms,
                          void *cuda_stream);
fpe_status fpe_batch_sync(fpe_batch_t B, void *cuda_stream);
void fpe_batch_destroy(fpe_batch_t B);
fpe_status fpe_eval_batch(const fpe_poly_t *P, int64_t npoly, const int64_t *pt_offsets, const double *z_re,
                          const double *z_im, fpe_xc64 *out, void *cuda_stream);

/*
 * Launch parameters of the window sums, and an autotuner for them (the paper
 * has no counterpart: they only schedule the same terms).
 *
 * A point whose window has more than long_window terms is summed by warp
 * groups: 32 lane chunks of at most lane_chunk terms each, combined by
 * shuffles, several groups per window when it is longer than 32 lane_chunk;
 * shorter windows take one thread each (32 points per warp).  Every setting
 * keeps the error bounds of fpe_eval; the order of the additions inside a
 * window changes, so values may differ in the last bits.  Defaults: 4096 and
 * 1024.
 *
 * fpe_set_tuning, fpe_batch_set_tuning: long_window in [32, 2^24],
 *   lane_chunk in [16, 2^16], else FPE_ERR_INVALID_ARG; t->ms is ignored.
 *   The setting applies to later evaluations of that handle or batch.
 * fpe_get_tuning: the handle's current setting (ms = 0 unless it came from
 *   fpe_autotune).
 * fpe_autotune: times fpe_eval on the caller's n device points (z_re, z_im
 *   as in fpe_eval) at every setting of the grid long_window in {1024, 2048,
 *   4096, 8192} x lane_chunk in {128, 256, 512, 1024, 2048}: one untimed call,
 *   then two calls between CUDA events on cuda_stream.  Keeps the fastest in
 *   the handle and returns it in *best (ms = its time per call).
 *   Synchronous; allocates and frees a temporary output array.  Errors as
 *   fpe_eval, FPE_ERR_INVALID_ARG for a NULL best.
 * fpe_batch_autotune: the same for a batch over its own points.
 */
typedef struct {
  int64_t long_window;
  int64_t lane_chunk;
  double ms;
} fpe_tuning;
fpe_status fpe_set_tuning(fpe_poly_t P, const fpe_tuning *t);
fpe_status fpe_get_tuning(fpe_poly_t P, fpe_tuning *t);
fpe_status fpe_autotune(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, void *cuda_stream,
                        fpe_tuning *best);
fpe_status fpe_batch_set_tuning(fpe_batch_t B, const fpe_tuning *t);
fpe_status fpe_batch_autotune(fpe_batch_t B, const double *z_re, const double *z_im, void *cuda_stream,
                              fpe_tuning *best);

/*
 * Tensor-core window sums (the same Q_lambda(z) of Alg. A_p, eq. reducedQlambda,
 * computed on another unit; the paper has no
 * counterpart).  In the FP64 default mode (not FPE_FP32, not FPE_ACCURATE),
 * fpe_eval sums every window of at least min_window terms that lies inside
 * one of the polynomial's longest (up to four) coefficient pieces with an
 * integer cover slope on the bf16 tensor cores (tcgen05.mma with fp32
 * accumulators in tensor memory): coefficients and point powers are cut into
 * exact 7-bit digits whose products are added exactly, and blocks of 32
 * terms are combined in 64-bit mantissas (folded into 128 bits every 128
 * blocks) and 128-bit fixed point across work items.  Points are grouped
 * about 112 at a time by log2|z| into tiles of up to 128; a group also sums
 * the terms of its neighbours' windows
 * (all of them below the window threshold), and a group whose |z| spread is
 * too wide for one shared scaling goes back to the FP64 kernels.  The error
 * stays below 2^-53.5 sum |a_k||z|^k.
 *
 * fpe_set_tensor_path: min_window in {0} or [32, 2^30]; 0 turns the path
 *   off.  Default 384 (below a few hundred terms the FP64 kernels are
 *   cheaper than building a point's slices), and by default only on calls
 *   of at least 32768 points (the path's planning is a fixed cost of about
 *   ten launches); a value set here applies to calls of every size.
 *   Applies to later fpe_eval calls of that handle (not to fpe_eval_noalloc,
 *   the batch or the gradient paths).
 *   FPE_ERR_INVALID_ARG for a NULL handle or a value out of range.
 * fpe_get_tensor_path: the handle's current min_window, and in *n_pieces the
 *   number of its pieces that qualify (0: the path never runs for it).
 */
fpe_status fpe_set_tensor_path(fpe_poly_t P, int64_t min_window);
fpe_status fpe_get_tensor_path(fpe_poly_t P, int64_t *min_window, int32_t *n_pieces);
/*
 * fpe_tensor_stats: what the tensor-core path did in the handle's last
 *   fpe_eval, in stats[0..5]: points it summed, tiles (up to 128 points that
 *   share a tilt and a block range), work items, MMA sub-tiles (8 blocks of
 *   32 terms by a tile's 128 point rows; each is 40 tcgen05.mma of M 128,
 *   K 16, N 16 (10 - s) for digit slice s, i.e. 1.44e7 bf16 flop), blocks
 *   per work item, and the points
 *   handed back to the FP64 kernels (their group's |z| spread too wide).
 *   All zero when the path did not run.  Waits for the work queued on
 *   cuda_stream.  FPE_ERR_INVALID_ARG for NULL arguments or n < 6.
 */
fpe_status fpe_tensor_stats(fpe_poly_t P, int64_t *stats, int n, void *cuda_stream);
/*
 * fpe_cert_stats: the rounding-error certificates of the handle's last
 *   fpe_eval (default FP64 mode), in stats[0]: the windows whose FP64 sum
 *   failed its certificate and was summed again exactly on the integer pipe.
 *   The default mode's values meet |P_gpu - P| <= 2^-50 sum |a_k||z|^k
 *   through these re-sums.  (Long windows, summed by warp groups, are summed
 *   exactly on the integer pipe in the first place.)  stats[1 .. n-1] are
 *   set to zero.  Zero for the other modes.  Waits for the work queued on
 *   cuda_stream.  FPE_ERR_INVALID_ARG for NULL arguments or n < 1.
 */
fpe_status fpe_cert_stats(fpe_poly_t P, int64_t *stats, int n, void *cuda_stream);

/*
 * fpe_newton -- one Newton step N_P(z) = z - P(z)/P'(z) (§7.2, eq. newton) at n
 * points.  P(z) and P'(z) are evaluated by the FPE path as extended-exponent
 * values, so the increment P/P' never overflows where P and P' do (the
 * paper's cancellation of the valuation monomial z^m, m = min(l, l'), gives
 * the same protection).  Requires FPE_WITH_DERIV.
 *   inc         device fpe_xc64[n]: P(z)/P'(z) (0 where P(z) = 0; NaN where only P' vanishes).
 *   z_next_re/im device double[n] or NULL: z - inc as FP64 (inf where inc overflows FP64).
 * Asynchronous; the first call allocates scratch on the handle.  P' is
 * evaluated on a second stream (one per device, created on first use and
 * kept until exit) beside P on cuda_stream, forked from and joined back into
 * cuda_stream, so the step is ordered on cuda_stream like any other call.
 */
fpe_status fpe_newton(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *inc,
                      double *z_next_re, double *z_next_im, void *cuda_stream);

/*
 * fpe_grad_points -- the gradient with respect to the points of a real loss L
 * of the values P(z_j): dL/dz_j = g_j conj(P'(z_j)) with g_j = dL/dP(z_j) (the
 * conjugate Wirtinger convention; P is holomorphic in z).  P' is evaluated by
 * the FPE path (§7.2).  Requires FPE_WITH_DERIV.  g_re/g_im (g_im NULL = real)
 * and gz_re/gz_im (gz_im may be NULL) are device double[n].  The gradient is
 * written in FP64: where g conj(P') leaves the FP64 range it is +-inf (or NaN
 * when an infinite part meets a zero one), and no status reports it; callers
 * that need those points take P' from fpe_eval_deriv, whose values carry
 * their own exponent.  Asynchronous.
 */
fpe_status fpe_grad_points(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, const double *g_re,
                           const double *g_im, double *gz_re, double *gz_im, void *cuda_stream);

/*
 * fpe_grad_coeffs -- ADDS to ga the gradient with respect to the coefficients:
 * dL/da_k += sum_j g_j conj(z_j)^k over the terms the evaluation kept,
 * k in G_p cap [l_j, r_j] (eq. reducedQlambda): the FPE value at z_j depends on
 * no other coefficient.  ga_re/ga_im are device double[n_coef] (untrimmed
 * index; ga_im may be NULL for a real polynomial).  Atomic accumulation:
 * the summation order, hence the last bits, vary between runs.  Asynchronous.
 */
fpe_status fpe_grad_coeffs(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, const double *g_re,
                           const double *g_im, double *ga_re, double *ga_im, void *cuda_stream);

/* fpe_to_complex -- (re, im) 2^e of n device fpe_xc64 values as device FP64
 * (inf or 0 where the value leaves the FP64 range); im may be NULL.  Async. */
fpe_status fpe_to_complex(const fpe_xc64 *v, int64_t n, double *re, double *im, void *cuda_stream);

/*
 * fpe_horner -- the plain form beside FPE: Horner's scheme over all d+1
 * coefficients (§1, "Horner's scheme") on the GPU, with exact power-of-two
 * renormalisation so that no intermediate overflows.
 *   compensated = 0: FP64 Horner (4 FMA per complex term).
 *   compensated = 1: compensated Horner with error-free transformations
 *                    (TwoSum, FMA TwoProd; the compensated schemes cited in
 *                    §1), about 2^-53 relative error plus a second-order term.
 * Arguments as fpe_eval (device pointers).  Asynchronous.
 */
fpe_status fpe_horner(fpe_poly_t P, const double *z_re, const double *z_im, int64_t n, fpe_xc64 *out,
                      int compensated, void *cuda_stream);

/* fpe_info -- degree d (last nonzero index), valuation v (first nonzero index),
 * number of cover vertices, |G_p|, and T = p + s(d) + 3.  Any output may be NULL. */
fpe_status fpe_info(fpe_poly_t P, int64_t *d, int64_t *valuation, int64_t *n_hull, int64_t *n_good, int *T);

/* fpe_get_hull -- the cover's vertices (k_i, s(a_{k_i})) in untrimmed indices,
 * left to right, strict vertices only.  k, s: host arrays of capacity cap >= n_hull. */
fpe_status fpe_get_hull(fpe_poly_t P, int64_t *k, int64_t *s, int64_t cap);

/* fpe_get_good -- G_p as a host 0/1 mask of n_coef bytes (untrimmed indices). */
fpe_status fpe_get_good(fpe_poly_t P, uint8_t *mask, int64_t n_coef);

/* fpe_get_windows -- the per-point data of the last fpe_eval on this handle,
 * for inspection: l, r (untrimmed; l > r for z = 0) and N (eq. defN), as
 * device arrays of n entries in the caller's point order.  Asynchronous. */
fpe_status fpe_get_windows(fpe_poly_t P, int64_t n, int64_t *l, int64_t *r, double *N, void *cuda_stream);

/*
 * fpe_analyse -- the |z|-ranges on which each coefficient is used (the
 * -analyse task of §8.1): a good coefficient k is kept, k in [l, r] (def. LRN),
 * exactly when lam_lo[k] <= log2|z| <= lam_hi[k] (the set is an interval
 * because cover(k) + lambda k - N(lambda) is concave in lambda; the ends are
 * +-inf when unbounded).  Bad coefficients (not in G_p) get NaN.  Host arrays
 * of n_coef doubles, untrimmed indices; FP64 endpoints (ties at an endpoint
 * may go either way, as in fpe_eval).  Works on FPE_HOST_ONLY handles.
 */
fpe_status fpe_analyse(fpe_poly_t P, double *lam_lo, double *lam_hi, int64_t n_coef);

/* fpe_sync -- wait for the stream and return the first device-side status
 * recorded on the handle since the last fpe_sync (then clear it). */
fpe_status fpe_sync(fpe_poly_t P, void *cuda_stream);

/* fpe_destroy -- free the handle and its device memory.  NULL is a no-op. */
void fpe_destroy(fpe_poly_t P);

/* fpe_status_string -- static description of a status code. */
const char *fpe_status_string(fpe_status s);

/* fpe_last_error -- thread-local message for the last failing call (static storage). */
const char *fpe_last_error(void);

/*
 * Kernel timing (measurement support, no counterpart in the paper).  When
 * enabled, every kernel launch of this library (or a short run of launches
 * of one stage under one name: k_tc_plan = k_tc_plan_a, _b, _c; k_tc_pre =
 * k_tc_tau, k_tc_pre; k_tc_finalize = its two launches) records CUDA events
 * around itself on its launching stream; fpe_profile_read() synchronises
 * with the events and returns, for names that contain `name`, the total
 * device time in milliseconds and the number of kernel launches since the
 * last reset.
 */
void fpe_profile_enable(int on);
void fpe_profile_reset(void);
fpe_status fpe_profile_read(const char *name, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* FPE_H_ */
