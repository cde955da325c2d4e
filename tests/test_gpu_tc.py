"""Tensor-core form (split-FP16 tcgen05 M2L, FP32 elsewhere) against the FP64
oracle: rel-l2 within the 1e-6 target on multi-level trees for every order
the form supports, plus the FP64 GPU form as a second reference."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from oracle.fdm import FDMOracle
from paper_2004_14229_gb300.workloads import complex_normal, uniform_points, workload
from tests.gpu_common import gpu_apply, rel_l2

pytestmark = pytest.mark.gpu

TOL_TC = 1e-6


def test_tc_small_workload_against_oracle():
    t, s, x, w = workload("uniform-8k-k16-d4-o4")
    o = FDMOracle(t, s, w["kappa"], w["order"], [0, 0, 0], 1.0, w["depth"])
    yo = o.apply(x)
    with pkg.Plan(t, s, w["kappa"], order=w["order"], max_depth=w["depth"],
                  precision=pkg.TC_FP16X3) as plan:
        y = gpu_apply(plan, x.astype(np.complex64))
        plan.check()
    err = rel_l2(y, yo)
    print("TC vs oracle rel l2 = %.3e" % err)
    assert err < TOL_TC


@pytest.mark.parametrize("n,kappa,order,depth", [
    (4000, 40.0, 3, 4),     # high-frequency leaves, 6 directions on the leaf level
    (5000, 24.0, 5, 4),
    (6000, 30.0, 6, 4),
    (3000, 20.0, 2, 3),
])
def test_tc_orders_against_oracle(n, kappa, order, depth):
    t = uniform_points(n, 21)
    s = uniform_points(n + 77, 22)
    x = complex_normal(n + 77, 23)
    o = FDMOracle(t, s, kappa, order, [0, 0, 0], 1.0, depth)
    with pkg.Plan(t, s, kappa, order=order, max_depth=depth, precision=pkg.TC_FP16X3) as plan:
        y = gpu_apply(plan, x.astype(np.complex64))
        plan.check()
    err = rel_l2(y, o.apply(x))
    print("order %d: TC vs oracle rel l2 = %.3e" % (order, err))
    assert err < TOL_TC


def test_tc_matches_fp64_form_and_is_deterministic():
    t = uniform_points(20000, 31)
    s = uniform_points(20000, 32)
    x = complex_normal(20000, 33)
    with pkg.Plan(t, s, 48.0, order=6, max_depth=5) as p64:
        y64 = gpu_apply(p64, x)
    with pkg.Plan(t, s, 48.0, order=6, max_depth=5, precision=pkg.TC_FP16X3) as ptc:
        ya = gpu_apply(ptc, x.astype(np.complex64))
        yb = gpu_apply(ptc, x.astype(np.complex64))
        ptc.check()
    err = rel_l2(ya, y64)
    print("TC vs FP64 form rel l2 = %.3e" % err)
    assert err < TOL_TC
    assert rel_l2(yb, ya) < 1e-6


def test_non_finite_input_reports_numeric_error():
    t = uniform_points(3000, 71)
    s = uniform_points(3000, 72)
    x = complex_normal(3000, 73).astype(np.complex64)
    x[5] = np.nan
    with pkg.Plan(t, s, 20.0, order=4, max_depth=3, precision=pkg.TC_FP16X3) as p:
        gpu_apply(p, x)
        with pytest.raises(pkg.DFDMError) as e:
            p.check()
        assert e.value.status == 5          # DFDM_ERR_NUMERIC
        # the check clears the word; a finite input runs clean again
        y = gpu_apply(p, complex_normal(3000, 74).astype(np.complex64))
        p.check()
        assert np.all(np.isfinite(y))


def test_tc_multi_rhs_matches_single_rhs_and_oracle():
    """Several right-hand sides at once (leaves of ~40 points: the nearfield of
    all right-hand sides runs as one pass, f(x, y) formed once per pair) equal
    the products of one right-hand side at a time, and the oracle's."""
    import torch
    n, nrhs = 20000, 10          # 10: one full group of 8 and a partial one
    t = uniform_points(n, 41)
    s = uniform_points(n, 42)
    xs = np.stack([complex_normal(n, 43 + r) for r in range(nrhs)])
    with pkg.Plan(t, s, 30.0, order=4, max_depth=3, precision=pkg.TC_FP16X3, nrhs_max=nrhs) as plan:
        assert plan.stats()["nf_entries"] > 0
        xd = torch.from_numpy(xs.astype(np.complex64)).cuda()
        y_all = plan.apply(xd).cpu().numpy()
        plan.check()
        for r in (0, 7, 8, 9):
            y_one = plan.apply(xd[r]).cpu().numpy()
            assert rel_l2(y_all[r], y_one) < 1e-6, r
    o = FDMOracle(t, s, 30.0, 4, [0, 0, 0], 1.0, 3)
    rows = np.arange(0, n, 97)
    for r in (0, 9):
        err = rel_l2(y_all[r][rows], o.apply(xs[r], rows=rows))
        print("multi-RHS TC vs oracle rel l2 (rhs %d) = %.3e" % (r, err))
        assert err < TOL_TC
