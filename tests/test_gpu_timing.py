"""Per-phase timing (dfdm_plan_set_timing / dfdm_plan_timing): the events of
consecutive applies accumulate without host synchronisation and one read
returns their sums."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from paper_2004_14229_gb300.workloads import complex_normal, uniform_points

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pkg.TC_FP16X3, pkg.FP64])
def test_timing_accumulates_until_read(precision):
    import torch
    t = uniform_points(30000, 61)
    x = complex_normal(30000, 62)
    dt = np.complex64 if precision == pkg.TC_FP16X3 else np.complex128
    xd = torch.from_numpy(x.astype(dt)).cuda()
    with pkg.Plan(t, t, 24.0, order=4, max_depth=4, precision=precision) as plan:
        y = plan.apply(xd)
        plan.set_timing(True)
        for _ in range(3):
            plan.apply(xd, y)
        a = plan.timing()
        assert a["applies"] == 3 and a["launches"] % 3 == 0 and a["launches"] > 0
        phases = a["s2m_ms"] + a["m2m_ms"] + a["split_ms"] + a["l2l_ms"] + a["l2t_ms"] + a["near_ms"]
        assert 0 < phases + sum(a["m2l_ms"]) <= a["total_ms"] * 1.001
        with pytest.raises(pkg.DFDMError) as e:    # nothing since the read
            plan.timing()
        assert e.value.status == 1
        plan.apply(xd, y)
        b = plan.timing()
        assert b["applies"] == 1 and b["launches"] == a["launches"] // 3
        assert b["total_ms"] < a["total_ms"]
        plan.set_timing(False)
        plan.check()
