"""Write the stored oracle values for the large workloads.

Calls only oracle/ (and the seeded input generators): for each named
workload, the exact direct sum (O_direct, Eq. 1) at `ndirect` sampled target
rows (sample_rows(n, ndirect, seed=4)) and the FP64 oracle's fast directional
product (Alg. 4, O_fdm) at every `stride`-th of those rows.  The GPU tests and
the benchmark compare the CUDA path against these values.

    python tests/golden/make_golden.py uniform-4M-k128-d7-o6 [nfdm [ndirect [out_dir]]]

nfdm rows of O_fdm are taken evenly from the ndirect direct-sum rows
(ndirect defaults to nfdm).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.direct import direct_rows, direct_threads  # noqa: E402
from oracle.fdm import FDMOracle  # noqa: E402
from paper_2004_14229_gb300.workloads import sample_rows, workload  # noqa: E402


def fdm_subset(rows_direct, nfdm):
    """The O_fdm rows: nfdm of the direct-sum rows, evenly spaced in the sorted sample."""
    nd = rows_direct.size
    pick = (np.arange(nfdm, dtype=np.int64) * nd) // max(nfdm, 1)
    return rows_direct[pick]


def main():
    name = sys.argv[1]
    nfdm = int(sys.argv[2]) if len(sys.argv) > 2 else 16
    ndirect = int(sys.argv[3]) if len(sys.argv) > 3 else nfdm
    out_dir = sys.argv[4] if len(sys.argv) > 4 else os.path.dirname(os.path.abspath(__file__))
    ndirect = max(ndirect, nfdm)
    t, s, x, w = workload(name)
    rows_dir = sample_rows(w["n"], ndirect, seed=4)
    rows = fdm_subset(rows_dir, nfdm)
    t0 = time.time()
    y_dir_all = direct_rows(t, s, w["kappa"], x, rows_dir)
    t1 = time.time()
    o = FDMOracle(t, s, w["kappa"], w["order"], [0, 0, 0], 1.0, w["depth"])
    y_fdm = o.apply(x, rows=rows)
    t2 = time.time()
    y_dir = y_dir_all[np.searchsorted(rows_dir, rows)]
    out = os.path.join(out_dir, "%s_rows.npz" % name)
    np.savez(out, rows=rows, y_fdm=y_fdm, y_direct=y_dir, rows_direct=rows_dir, y_direct_all=y_dir_all,
             l_hf=o.l_hf,
             note=np.array("O_direct at sample_rows(n, %d, seed=4); O_fdm (Alg. 4, FP64, reuse mode) at %d of "
                           "them, evenly spaced" % (ndirect, nfdm)))
    print("%s: %d direct rows (%.1f s, %d threads), %d O_fdm rows (%.1f s), rel err O_fdm vs O_direct %.3e -> %s"
          % (name, ndirect, t1 - t0, direct_threads(), nfdm, t2 - t1,
             np.linalg.norm(y_fdm - y_dir) / np.linalg.norm(y_dir), out))


if __name__ == "__main__":
    main()
