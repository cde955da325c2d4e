"""Batched form (dfdm_batch_*): every problem's result equals its own plan's
product, and the oracle's on sampled rows; graph replays repeat the result."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from oracle.fdm import FDMOracle
from paper_2004_14229_gb300.workloads import batch_problems, sample_rows
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu

ROOT = ((0.0, 0.0, 0.0), 1.0)


def _problems():
    # uniform, Gaussian and shell problems of 2k .. 12k points, kappa 4 .. 40
    return batch_problems(6, n_range=(2000, 12000), kappa_range=(4.0, 40.0), nrhs=2, seed0=300)


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.TC_FP16X3])
def test_batch_matches_single_plans_and_oracle(precision):
    import torch
    probs = _problems()
    dt = torch.complex128 if precision == pkg.FP64 else torch.complex64
    tol_plan = 1e-13 if precision == pkg.FP64 else 1e-6
    tol_oracle = 1e-10 if precision == pkg.FP64 else 1e-6
    batch = pkg.Batch(probs, order=4, root=ROOT, precision=precision, nrhs_max=2, nstreams=3)
    try:
        xs = [torch.from_numpy(p["x"]).to(dtype=dt, device="cuda") for p in probs]
        ys = [torch.empty((2, p["targets"].shape[0]), dtype=dt, device="cuda") for p in probs]
        batch.apply(xs, ys)
        torch.cuda.synchronize()
        batch.check()
        first = [y.cpu().numpy().copy() for y in ys]
        ns, stream_of, launches = batch.info()
        assert ns == 3 and set(stream_of.tolist()) <= {0, 1, 2} and launches > 0
        # replay of the captured graph (same pointers) repeats the product
        batch.apply(xs, ys)
        torch.cuda.synchronize()
        for a, y in zip(first, ys):
            assert rel_l2(y.cpu().numpy(), a) < tol_plan
        for i, p in enumerate(probs):
            with pkg.Plan(p["targets"], p["sources"], p["kappa"], order=4, max_depth=p["max_depth"],
                          root=ROOT, precision=precision, nrhs_max=2) as plan:
                ref = plan.apply(xs[i])
                torch.cuda.synchronize()
                assert rel_l2(first[i], ref.cpu().numpy()) < tol_plan, i
        for i in (1, 2):   # a Gaussian and a shell problem against the oracle
            p = probs[i]
            rows = sample_rows(p["targets"].shape[0], 200, seed=7 + i)
            o = FDMOracle(p["targets"], p["sources"], p["kappa"], 4, ROOT[0], ROOT[1], p["max_depth"])
            for r in range(2):
                want = o.apply(p["x"][r], rows=rows)
                assert rel_l2(first[i][r][rows], want) < tol_oracle, (i, r)
    finally:
        batch.close()


def test_batch_new_pointers_recapture():
    import torch
    probs = _problems()[:3]
    batch = pkg.Batch(probs, order=3, root=ROOT, precision=pkg.TC_FP16X3, nrhs_max=2, nstreams=2)
    try:
        xs = [torch.from_numpy(p["x"][:1]).to(dtype=torch.complex64, device="cuda") for p in probs]
        ya = [torch.empty((1, p["targets"].shape[0]), dtype=torch.complex64, device="cuda") for p in probs]
        yb = [torch.empty((1, p["targets"].shape[0]), dtype=torch.complex64, device="cuda") for p in probs]
        batch.apply(xs, ya)
        batch.apply(xs, yb)     # other output pointers: a new graph
        torch.cuda.synchronize()
        batch.check()
        for a, b in zip(ya, yb):
            assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) < 1e-6
    finally:
        batch.close()
