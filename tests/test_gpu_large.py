"""The products at the benchmark's sizes against stored FP64 oracle rows
(tests/golden/*_rows.npz, written by tests/golden/make_golden.py from the
oracle alone), in the launch configuration bench.py times."""
import os

import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from paper_2004_14229_gb300.workloads import workload
from tests.gpu_common import gpu_apply, rel_l2

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    return np.load(os.path.join(GOLD, "%s_rows.npz" % name))


@pytest.mark.parametrize("name,precision,tol", [
    ("uniform-1M-k64-d6-o5", pkg.FP64, 1e-10),
    ("uniform-1M-k64-d6-o5", pkg.TC_FP16X3, 1e-6),
    ("uniform-4M-k128-d7-o6", pkg.TC_FP16X3, 1e-6),
])
def test_full_size_rows_against_oracle(name, precision, tol):
    t, s, x, w = workload(name)
    g = _golden(name)
    with pkg.Plan(t, s, w["kappa"], order=w["order"], max_depth=w["depth"], precision=precision) as plan:
        st = plan.stats()
        assert st["l_hf"] == int(g["l_hf"])
        xin = x if precision == pkg.FP64 else x.astype(np.complex64)
        y = gpu_apply(plan, xin)
        plan.check()
    err = rel_l2(y[g["rows"]], g["y_fdm"])
    # the method's own error against the exact sum is the oracle's
    err_dir = rel_l2(y[g["rows"]], g["y_direct"])
    err_dir_oracle = rel_l2(g["y_fdm"], g["y_direct"])
    print("%s %s: vs O_fdm %.3e, vs O_direct %.3e (oracle %.3e)" % (name, precision, err, err_dir, err_dir_oracle))
    assert err < tol
    assert abs(err_dir - err_dir_oracle) < 10 * tol + 1e-12
