"""The products at the benchmark's sizes against stored FP64 oracle rows
(tests/golden/*_rows.npz, written by tests/golden/make_golden.py from the
oracle alone: O_fdm at 128 / 256 rows, the exact direct sum at 2048 rows), in
the launch configuration bench.py times."""
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


def _plan(name, precision):
    t, s, x, w = workload(name)
    plan = pkg.Plan(t, s, w["kappa"], order=w["order"], max_depth=w["depth"], precision=precision)
    xin = x if precision == pkg.FP64 else x.astype(np.complex64)
    return plan, xin


def _check_rows(name, y, tol, g):
    err = rel_l2(y[g["rows"]], g["y_fdm"])
    # the method's own error against the exact sum is the oracle's ("equal accuracy")
    err_dir = rel_l2(y[g["rows"]], g["y_direct"])
    err_dir_oracle = rel_l2(g["y_fdm"], g["y_direct"])
    err_dir_all = rel_l2(y[g["rows_direct"]], g["y_direct_all"])
    print("%s: vs O_fdm (%d rows) %.3e; vs O_direct %.3e (oracle %.3e); vs O_direct on %d rows %.3e"
          % (name, g["rows"].size, err, err_dir, err_dir_oracle, g["rows_direct"].size, err_dir_all))
    assert err < tol
    assert abs(err_dir - err_dir_oracle) < 10 * tol + 1e-12
    return err, err_dir_all


def test_1m_fp64_and_tensor_core_forms():
    """1M points, kappa 64, order 5: the FP64 form within 1e-10 of the oracle
    rows; the tensor-core form within 1e-6 of the oracle rows AND of the FP64
    form over all 2^20 rows."""
    name = "uniform-1M-k64-d6-o5"
    g = _golden(name)
    plan, xin = _plan(name, pkg.FP64)
    with plan:
        assert plan.stats()["l_hf"] == int(g["l_hf"])
        y64 = gpu_apply(plan, xin)
        plan.check()
    _check_rows(name + " FP64", y64, 1e-10, g)
    plan, xin = _plan(name, pkg.TC_FP16X3)
    with plan:
        ytc = gpu_apply(plan, xin)
        plan.check()
    _check_rows(name + " TC", ytc, 1e-6, g)
    err_all = rel_l2(ytc, y64)
    print("%s: TC vs FP64 form over all %d rows %.3e" % (name, ytc.size, err_all))
    assert err_all < 1e-6


def test_4m_tensor_core_form_rows_against_oracle():
    """The benchmark workload (2^22 points, kappa 128, depth 7, order 6):
    the tensor-core form within 1e-6 of 256 oracle rows, with the built-in
    launch shapes and with the tuned ones bench.py times."""
    import torch
    name = "uniform-4M-k128-d7-o6"
    g = _golden(name)
    plan, xin = _plan(name, pkg.TC_FP16X3)
    with plan:
        assert plan.stats()["l_hf"] == int(g["l_hf"])
        y = gpu_apply(plan, xin)
        plan.check()
        plan.autotune(torch.from_numpy(xin).cuda())
        y_tuned = gpu_apply(plan, xin)
        plan.check()
    _check_rows(name + " TC", y, 1e-6, g)
    _check_rows(name + " TC, tuned launch shapes", y_tuned, 1e-6, g)
