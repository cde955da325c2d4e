"""The FP32 nearfield on large leaves (the blocks of k_p2p_f32: 128-thread
blocks, and one-warp blocks over several target chunks of a leaf, ragged
last chunks; k_p2p_mrhs for several right-hand sides) against the exact
direct sum of Eq. (1) computed by the oracle on sampled rows, and against the
FP64 GPU form (itself held to 1e-10 of the oracle) over all rows."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from oracle.direct import direct_rows
from paper_2004_14229_gb300.workloads import complex_normal, sample_rows, tensor_grid, uniform_points
from tests.gpu_common import gpu_apply, rel_l2

pytestmark = pytest.mark.gpu


def _case(kind):
    if kind == "grid-k5":        # Sect. 4's grid: P_S = P_T, 64 leaves of 512 points, zero diagonal
        t = tensor_grid(5)
        return t, t, 3.2, dict(order=5, max_depth=8, n_max=512, root=((-1.0, -1.0, -1.0), 2.0))
    if kind == "uniform-d2":     # 64 leaves of ~780 points: seven target chunks, the last one ragged
        return (uniform_points(50000, 41), uniform_points(48000, 42), 12.0,
                dict(order=4, max_depth=2))
    # 4096 leaves of ~73 points: one 128-thread block per leaf
    return uniform_points(300000, 43), uniform_points(300000, 44), 20.0, dict(order=4, max_depth=4)


@pytest.mark.parametrize("kind", ["grid-k5", "uniform-d2", "uniform-d4"])
def test_fp32_nearfield_on_large_leaves(kind):
    t, s, kappa, kw = _case(kind)
    x = complex_normal(s.shape[0], 45)
    rows = sample_rows(t.shape[0], 96, seed=46)
    yd = direct_rows(t, s, kappa, x, rows)
    with pkg.Plan(t, s, kappa, precision=pkg.FP64, **kw) as plan:
        y64 = gpu_apply(plan, x)
        plan.check()
    with pkg.Plan(t, s, kappa, precision=pkg.TC_FP16X3, **kw) as plan:
        ytc = gpu_apply(plan, x.astype(np.complex64))
        plan.check()
    e_all = rel_l2(ytc, y64)
    e_tc, e_64 = rel_l2(ytc[rows], yd), rel_l2(y64[rows], yd)
    print("%s: TC vs FP64 form %.3e; vs O_direct rows TC %.3e FP64 %.3e" % (kind, e_all, e_tc, e_64))
    assert e_all < 1e-6
    # same approximation error against the exact sum, up to the FP32 rounding
    assert abs(e_tc - e_64) < 1e-6


def test_fp32_nearfield_several_rhs_on_large_leaves():
    t, s, kappa, kw = _case("grid-k5")
    xs = complex_normal(s.shape[0], 47, nrhs=5).astype(np.complex64)
    import torch
    with pkg.Plan(t, s, kappa, precision=pkg.TC_FP16X3, nrhs_max=5, **kw) as plan:
        y_all = plan.apply(torch.from_numpy(xs).cuda()).cpu().numpy()
        for r in range(5):
            y_one = gpu_apply(plan, xs[r])
            assert rel_l2(y_all[r], y_one) < 1e-6, r
        plan.check()
