/*
 * O_direct: the exact matrix-vector product y = A x of Eq. (1), in FP64.
 *
 * TEST INFRASTRUCTURE ONLY. This file is part of the CPU oracle; it is built
 * and called by the tests, by the smoke check and by the CPU-baseline leg of
 * the benchmark, never by the library's product path. It shares no code with
 * the CUDA path.
 *
 * A[j,k] = f(x_j, y_k),  f(x,y) = exp(i kappa |x-y|) / (4 pi |x-y|)   (Eq. 1)
 *
 * Where a target coincides bit for bit with a source the entry is taken as 0
 * (Sect. 4 sets the diagonal of A to zero for P_S = P_T; the same rule is used
 * for any coincident pair).
 *
 * Layout: points are N x 3 row-major doubles; x and y are interleaved complex
 * (re, im) doubles.  Only the rows listed in `rows` are evaluated; y receives
 * them in the order of `rows` (y has 2*nrows doubles).  Each row is a plain
 * sequential sum over k = 0 .. n_s-1.
 */
#include <math.h>
#include <stdint.h>

#define ORACLE_PI 3.14159265358979323846

void oracle_direct_rows(const double *tgt, int64_t n_t, const double *src,
                        int64_t n_s, double kappa, const double *x,
                        const int64_t *rows, int64_t nrows, double *y) {
  (void)n_t;
  const double inv4pi = 1.0 / (4.0 * ORACLE_PI);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t j = rows[r];
    const double xj0 = tgt[3 * j + 0], xj1 = tgt[3 * j + 1],
                 xj2 = tgt[3 * j + 2];
    double acc_re = 0.0, acc_im = 0.0;
    for (int64_t k = 0; k < n_s; ++k) {
      const double y0 = src[3 * k + 0], y1 = src[3 * k + 1],
                   y2 = src[3 * k + 2];
      if (xj0 == y0 && xj1 == y1 && xj2 == y2) continue; /* zero diagonal */
      const double d0 = xj0 - y0, d1 = xj1 - y1, d2 = xj2 - y2;
      const double rr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      const double s = inv4pi / rr;
      const double f_re = cos(kappa * rr) * s;
      const double f_im = sin(kappa * rr) * s;
      const double xr = x[2 * k], xi = x[2 * k + 1];
      acc_re += f_re * xr - f_im * xi;
      acc_im += f_re * xi + f_im * xr;
    }
    y[2 * r] = acc_re;
    y[2 * r + 1] = acc_im;
  }
}

/* Number of OpenMP threads the routine above uses (1 without OpenMP). */
int oracle_direct_threads(void) {
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    {
#ifdef _OPENMP
      extern int omp_get_num_threads(void);
      n = omp_get_num_threads();
#endif
    }
  }
  return n;
}
