"""Sect. 4's workload on the GPU at the sizes the oracle cannot reach: the
8^k-point tensor grid (P_S = P_T, n_max = 512, kappa = 0.1 2^k, m = 4, i.e.
order 5).  The plan's counters equal Table 1's printed N_C, N_SC and
nearfield share (tests/golden/table1.json), and the product's error against
exact rows of Eq. (1) (the library's FP64 direct-sum kernel, itself held to
the oracle's direct sum in test_gpu_direct.py) is the method's approximation
error, of the size Sect. 4 reports (2e-4 at k = 6, m = 4)."""
import json
import os

import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from paper_2004_14229_gb300.workloads import sample_rows, workload
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu
TABLE = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1.json")))


@pytest.mark.parametrize("k", [6, 8])
def test_paper_grid_counts_and_error(k):
    import torch
    t, s, x, w = workload("paper-grid-k%d" % k)
    row = TABLE["rows"][str(k)]
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    with pkg.Plan(t, s, w["kappa"], order=w["order"], max_depth=w["depth"], n_max=w["n_max"], root=w["root"],
                  precision=pkg.TC_FP16X3) as plan:
        st = plan.stats()
        assert (st["depth"], st["l_hf"]) == (k - 3, k - 4)
        assert st["n_coupling"] == row["N_C"] and st["n_stored_coupling"] == row["N_SC"]
        digits = len(str(row["nf_percent"]).split(".")[1])
        assert round(100.0 * st["nf_entries"] / float(row["N"]) ** 2, digits) == pytest.approx(row["nf_percent"])
        y = plan.apply(xd).cpu().numpy()
        plan.check()
    rows = sample_rows(w["n"], 64, seed=4)
    td = torch.from_numpy(t).cuda()
    want = pkg.direct_rows(td, td, w["kappa"], torch.from_numpy(x).cuda(), torch.from_numpy(rows).cuda())
    err = rel_l2(y[rows].astype(np.complex128), want.cpu().numpy())
    print("k = %d: rel-l2 against exact rows %.3e (Sect. 4: %.0e at k = 6)" % (k, err, TABLE["relative_error_k6_m4"]))
    assert err < 1e-3
