"""The stored oracle rows (tests/golden/*_rows.npz) still belong to the
workloads they were written for: the row indices are the seeded sample (the
O_fdm rows an even subset of the direct-sum rows), the exact direct-sum values
are recomputed here by the oracle on a subset, and the stored fast-method
values sit within the method's approximation error of them."""
import os

import numpy as np
import pytest

from oracle.direct import direct_rows
from oracle.fdm import default_l_hf
from paper_2004_14229_gb300.workloads import sample_rows, workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fdm_subset(rows_direct, nfdm):
    pick = (np.arange(nfdm, dtype=np.int64) * rows_direct.size) // nfdm
    return rows_direct[pick]


@pytest.mark.parametrize("name,approx,nfdm", [("uniform-1M-k64-d6-o5", 5e-3, 128),
                                              ("uniform-4M-k128-d7-o6", 2e-3, 256)])
def test_golden_rows_match_workload_and_oracle(name, approx, nfdm):
    g = np.load(os.path.join(GOLDEN, "%s_rows.npz" % name))
    t, s, x, w = workload(name)
    rows, rows_dir = g["rows"], g["rows_direct"]
    assert rows.size == nfdm and rows_dir.size == 2048
    assert np.array_equal(rows_dir, sample_rows(w["n"], 2048, seed=4))
    assert np.array_equal(rows, _fdm_subset(rows_dir, nfdm))
    assert int(g["l_hf"]) == default_l_hf(w["kappa"], 1.0, w["depth"])
    # the direct sums at the O_fdm rows are the stored 2048-row values there
    assert np.array_equal(g["y_direct"], g["y_direct_all"][np.searchsorted(rows_dir, rows)])
    # recompute a spread subset of the direct sums
    sub = rows_dir[::64]
    y = direct_rows(t, s, w["kappa"], x, sub)
    assert np.allclose(y, g["y_direct_all"][::64], rtol=1e-12, atol=0)
    err = np.linalg.norm(g["y_fdm"] - g["y_direct"]) / np.linalg.norm(g["y_direct"])
    assert 1e-6 < err < approx          # an approximation, not a copy of the direct sum


def test_golden_writer_runs_on_the_small_workload(tmp_path):
    import subprocess
    import sys
    script = os.path.join(GOLDEN, "make_golden.py")
    r = subprocess.run([sys.executable, script, "uniform-8k-k16-d4-o4", "6", "24", str(tmp_path)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    g = np.load(str(tmp_path / "uniform-8k-k16-d4-o4_rows.npz"))
    t, s, x, w = workload("uniform-8k-k16-d4-o4")
    assert np.array_equal(g["rows_direct"], sample_rows(w["n"], 24, seed=4))
    assert np.array_equal(g["rows"], _fdm_subset(g["rows_direct"], 6))
    assert np.allclose(g["y_direct_all"], direct_rows(t, s, w["kappa"], x, g["rows_direct"]), rtol=1e-12, atol=0)
    err = np.linalg.norm(g["y_fdm"] - g["y_direct"]) / np.linalg.norm(g["y_direct"])
    assert err < 1e-2
