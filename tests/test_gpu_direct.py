"""GPU direct summation (dfdm_direct_rows) against the oracle's O_direct."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from oracle.direct import direct_rows
from paper_2004_14229_gb300.workloads import complex_normal, sample_rows, uniform_points
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nt,ns,nrows", [(20000, 30000, 300), (50, 5000, 50), (3000, 7, 3000)])
def test_direct_rows_against_oracle(nt, ns, nrows):
    import torch
    t = uniform_points(nt, 41)
    s = uniform_points(ns, 42)
    s[:5] = t[:5]                        # coincident pairs contribute 0
    x = complex_normal(ns, 43)
    rows = sample_rows(nt, nrows, 44)
    y = pkg.direct_rows(torch.from_numpy(t).cuda(), torch.from_numpy(s).cuda(), 17.0,
                        torch.from_numpy(x).cuda(), torch.from_numpy(rows).cuda()).cpu().numpy()
    assert rel_l2(y, direct_rows(t, s, 17.0, x, rows)) < 1e-12


def test_direct_rows_out_of_range_row_is_nan():
    import torch
    t = uniform_points(100, 1)
    x = complex_normal(100, 2)
    rows = torch.tensor([3, 100, -1, 7], dtype=torch.int64, device="cuda")
    y = pkg.direct_rows(torch.from_numpy(t).cuda(), torch.from_numpy(t).cuda(), 5.0,
                        torch.from_numpy(x).cuda(), rows).cpu().numpy()
    assert np.isfinite(y[[0, 3]]).all() and np.isnan(y[[1, 2]].real).all()
