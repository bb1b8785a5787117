/* Coefficients of the Mandelbrot iterate p_n (p_0 = c, p_{k+1} = p_k^2 + c,
 * degree 2^n) as extended-exponent FP64: a_k = m_k 2^e_k with m_k in [0.5, 1)
 * or m_k = 0.  Input generator for the benchmark's Mandelbrot workload (no
 * part of the evaluation method); the Python version in __init__.py is the
 * definition, this one scales it to n = 20.
 *
 * Each squaring is a direct convolution of positive terms:
 *   out_k = sum_j a_j a_{k-j}.
 * The log-magnitudes e_j of the coefficients form a hump that is concave to
 * within a bit (checked at n <= 12), so the exponents e_j + e_{k-j} fall off
 * on both sides of their maximum near j = k/2.  Each output scans outward
 * from the middle and stops on a side once kStop consecutive terms lie more
 * than kDrop bits below the largest exponent seen: the terms left out are
 * each below 2^-kDrop of the output, at most 2^(n+1) of them, so the output
 * keeps its relative precision to 2^(-kDrop + n + 1) beyond the FP64
 * rounding of the sum.  Outputs are independent: OpenMP over k. */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { kDrop = 128, kStop = 16 };

static void square(const double *m, const int64_t *e, int64_t D, double *om, int64_t *oe) {
  const int64_t DD = 2 * D;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t k = 0; k <= DD; ++k) {
    const int64_t jmin = k - D > 0 ? k - D : 0, jmax = k < D ? k : D;
    const int64_t c = k / 2 < jmin ? jmin : (k / 2 > jmax ? jmax : k / 2);
    int64_t G = INT64_MIN, lo = c, hi = c;
    /* pass 1: the scanned range and the largest exponent in it */
    for (int dir = -1; dir <= 1; dir += 2) {
      int run = 0;
      for (int64_t j = dir < 0 ? c : c + 1; j >= jmin && j <= jmax; j += dir) {
        if (m[j] != 0.0 && m[k - j] != 0.0) {
          const int64_t x = e[j] + e[k - j];
          if (x > G) G = x;
          run = (G != INT64_MIN && x < G - kDrop) ? run + 1 : 0;
        } else {
          ++run;
        }
        if (dir < 0) lo = j; else hi = j;
        if (run >= kStop && G != INT64_MIN) break;
      }
    }
    if (G == INT64_MIN) {
      om[k] = 0.0;
      oe[k] = 0;
      continue;
    }
    /* pass 2: the scaled sum */
    double s = 0.0;
    for (int64_t j = lo; j <= hi; ++j) {
      if (m[j] == 0.0 || m[k - j] == 0.0) continue;
      const int64_t x = e[j] + e[k - j] - G;
      if (x < -1000) continue;
      s += ldexp(m[j] * m[k - j], (int)x);
    }
    int f;
    om[k] = frexp(s, &f);
    oe[k] = G + f;
  }
}

/* m_out, e_out: 2^n + 1 entries each.  Returns 0, or -1 when out of memory. */
int mandel_coeffs(int n, double *m_out, int64_t *e_out) {
  const int64_t N = ((int64_t)1 << n) + 1;
  double *m = (double *)calloc((size_t)N, sizeof(double)), *om = (double *)calloc((size_t)N, sizeof(double));
  int64_t *e = (int64_t *)calloc((size_t)N, sizeof(int64_t)), *oe = (int64_t *)calloc((size_t)N, sizeof(int64_t));
  if (!m || !om || !e || !oe) {
    free(m); free(om); free(e); free(oe);
    return -1;
  }
  m[1] = 0.5; /* p_0 = c: a_1 = 1 = 0.5 2^1 */
  e[1] = 1;
  int64_t D = 1;
  for (int it = 0; it < n; ++it) {
    square(m, e, D, om, oe);
    D *= 2;
    /* + c */
    if (om[1] == 0.0) {
      om[1] = 0.5;
      oe[1] = 1;
    } else {
      int f;
      const double s = om[1] + ldexp(1.0, (int)-oe[1]);
      om[1] = frexp(s, &f);
      oe[1] += f;
    }
    memcpy(m, om, (size_t)(D + 1) * sizeof(double));
    memcpy(e, oe, (size_t)(D + 1) * sizeof(int64_t));
  }
  memcpy(m_out, m, (size_t)N * sizeof(double));
  memcpy(e_out, e, (size_t)N * sizeof(int64_t));
  free(m); free(om); free(e); free(oe);
  return 0;
}
