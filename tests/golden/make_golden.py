"""Write the stored oracle values for the large workloads.

Calls only oracle/ (and the seeded input generators): for each named
workload, the FP64 oracle's fast directional product (Alg. 4, O_fdm) and the
exact direct sum (O_direct) at a few sampled target rows.  The GPU tests and
the benchmark compare the CUDA path against these values.

    python tests/golden/make_golden.py uniform-4M-k128-d7-o6 [nrows [out_dir]]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.direct import direct_rows  # noqa: E402
from oracle.fdm import FDMOracle  # noqa: E402
from paper_2004_14229_gb300.workloads import sample_rows, workload  # noqa: E402


def main():
    name = sys.argv[1]
    nrows = int(sys.argv[2]) if len(sys.argv) > 2 else 16
    out_dir = sys.argv[3] if len(sys.argv) > 3 else os.path.dirname(os.path.abspath(__file__))
    t, s, x, w = workload(name)
    rows = sample_rows(w["n"], nrows, seed=4)
    t0 = time.time()
    o = FDMOracle(t, s, w["kappa"], w["order"], [0, 0, 0], 1.0, w["depth"])
    y_fdm = o.apply(x, rows=rows)
    t1 = time.time()
    y_dir = direct_rows(t, s, w["kappa"], x, rows)
    out = os.path.join(out_dir, "%s_rows.npz" % name)
    np.savez(out, rows=rows, y_fdm=y_fdm, y_direct=y_dir, l_hf=o.l_hf,
             note=np.array("O_fdm (Alg. 4, FP64, reuse mode) and O_direct at rows sample_rows(n, %d, seed=4)" % nrows))
    print("%s: %d rows, O_fdm %.1f s, rel err O_fdm vs O_direct %.3e -> %s"
          % (name, nrows, t1 - t0, np.linalg.norm(y_fdm - y_dir) / np.linalg.norm(y_dir), out))


if __name__ == "__main__":
    main()
