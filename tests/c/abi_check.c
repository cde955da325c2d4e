/* Plain-C use of include/dfdm.h (no C++, no CUDA headers): the calls that
 * need no GPU.  Prints one line per check; exits non-zero on a failure. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "dfdm.h"

static int fails = 0;

static void check(int ok, const char *what) {
  printf("%s %s\n", ok ? "ok  " : "FAIL", what);
  if (!ok) ++fails;
}

int main(void) {
  dfdm_params p;
  double pts[6] = {0.1, 0.2, 0.3, 0.4, 0.5, 0.6};
  dfdm_plan plan = (dfdm_plan)1;
  dfdm_batch batch = (dfdm_batch)1;
  dfdm_problem prob;
  float feat[4];

  check(dfdm_version() != NULL && strlen(dfdm_version()) > 0, "dfdm_version");
  check(dfdm_params_default(&p) == DFDM_OK && p.order == 5 && p.max_depth == 6 && p.eta2 == 5.0 &&
            p.l_hf == -2 && p.precision == DFDM_FP64 && p.nrhs_max == 1,
        "dfdm_params_default");
  check(dfdm_params_default(NULL) == DFDM_ERR_INVALID_ARG, "params NULL");
  check(dfdm_plan_create(pts, 2, pts, 2, -1.0, &p, NULL, &plan) == DFDM_ERR_INVALID_ARG && plan == NULL,
        "kappa <= 0 rejected, *out cleared");
  check(strlen(dfdm_last_error()) > 0, "dfdm_last_error after a failure");
  p.order = 11;
  check(dfdm_plan_create(pts, 2, pts, 2, 1.0, &p, NULL, &plan) == DFDM_ERR_INVALID_ARG, "order 11 rejected");
  p.order = 7;
  p.precision = DFDM_TC_FP16X3;
  check(dfdm_plan_create(pts, 2, pts, 2, 1.0, &p, NULL, &plan) == DFDM_ERR_UNSUPPORTED,
        "tensor-core form above order 6 unsupported");
  check(dfdm_plan_destroy(NULL) == DFDM_OK, "destroy NULL");
  check(dfdm_apply(NULL, NULL, NULL, 1, NULL) == DFDM_ERR_INVALID_ARG, "apply NULL plan");
  dfdm_params_default(&p);
  p.n_max = 4;
  prob.targets = pts;
  prob.n_t = 2;
  prob.sources = pts;
  prob.n_s = 2;
  prob.kappa = 1.0;
  prob.max_depth = -1;
  check(dfdm_batch_create(1, &prob, &p, 0, NULL, &batch) == DFDM_ERR_INVALID_ARG && batch == NULL,
        "batch with n_max > 0 rejected");
  check(dfdm_batch_destroy(NULL) == DFDM_OK, "batch destroy NULL");
  check(dfdm_selector_param_count() == 8770, "selector parameter count");
  check(dfdm_selector_features(10.0, 1.0, 2, 4096, 1e-4, feat) == DFDM_OK &&
            fabs(feat[0] - 0.2f) < 1e-6 && fabs(feat[2] - log2(1.0 + 64.0) / 16.0) < 1e-6 &&
            fabs(feat[3] - 0.4f) < 1e-6,
        "selector features");
  {
    /* the rank-1 4 x 3 complex matrix a[i][j] = ((i + 1) + i I) (j + 1), as interleaved
       (re, im) doubles; its ACA reproduces it */
    double a[24], u[24], v[18];
    int rank = -1, i, j, l;
    for (i = 0; i < 4; ++i)
      for (j = 0; j < 3; ++j) {
        a[2 * (3 * i + j)] = (double)((i + 1) * (j + 1));
        a[2 * (3 * i + j) + 1] = (double)(i * (j + 1));
      }
    check(dfdm_aca(a, 4, 3, 1e-12, 3, u, v, &rank) == DFDM_OK && rank >= 1 && rank <= 2, "aca runs");
    {
      double err = 0.0, nrm = 0.0;
      for (i = 0; i < 4; ++i)
        for (j = 0; j < 3; ++j) {
          double re = 0.0, im = 0.0; /* sum_l u[i][l] conj(v[j][l]) */
          for (l = 0; l < 3; ++l) {
            const double ur = u[2 * (3 * i + l)], ui = u[2 * (3 * i + l) + 1];
            const double vr = v[2 * (3 * j + l)], vi = -v[2 * (3 * j + l) + 1];
            re += ur * vr - ui * vi;
            im += ur * vi + ui * vr;
          }
          err += (re - a[2 * (3 * i + j)]) * (re - a[2 * (3 * i + j)]) +
                 (im - a[2 * (3 * i + j) + 1]) * (im - a[2 * (3 * i + j) + 1]);
          nrm += a[2 * (3 * i + j)] * a[2 * (3 * i + j)] + a[2 * (3 * i + j) + 1] * a[2 * (3 * i + j) + 1];
        }
      check(sqrt(err) <= 1e-12 * sqrt(nrm), "aca reproduces a low-rank matrix");
    }
    check(dfdm_aca(NULL, 4, 3, 1e-12, 3, u, v, &rank) == DFDM_ERR_INVALID_ARG, "aca NULL matrix");
    check(dfdm_plan_autotune(NULL, NULL, NULL, NULL, NULL) == DFDM_ERR_INVALID_ARG, "autotune NULL plan");
  }
  return fails != 0;
}
