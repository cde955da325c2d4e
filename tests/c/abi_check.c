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
  return fails != 0;
}
