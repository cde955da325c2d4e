"""dfdm_apply does no host synchronisation, so a product can be captured in a
CUDA graph (torch.cuda.CUDAGraph) and replayed; replays equal eager applies
(to rounding in the tensor-core form, whose coarse M2L levels split every
operator list over several CTAs that add into the locals atomically, so the
FP32 summation order differs from run to run)."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from paper_2004_14229_gb300.workloads import complex_normal, uniform_points
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.TC_FP16X3])
def test_apply_captured_in_cuda_graph(precision):
    import torch
    t = uniform_points(6000, 61)
    s = uniform_points(6000, 62)
    dt = torch.complex128 if precision == pkg.FP64 else torch.complex64
    x0 = torch.from_numpy(complex_normal(6000, 63)).to(dtype=dt, device="cuda")
    x1 = torch.from_numpy(complex_normal(6000, 64)).to(dtype=dt, device="cuda")
    with pkg.Plan(t, s, 30.0, order=4, max_depth=4, precision=precision) as plan:
        xin = x0.clone()
        yout = torch.empty(6000, dtype=dt, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            plan.apply(xin, yout, stream=side)        # warm-up on the capture stream
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.apply(xin, yout, stream=torch.cuda.current_stream())
        for x in (x0, x1, x0):
            xin.copy_(x)
            g.replay()
            torch.cuda.synchronize()
            ref = plan.apply(x)
            torch.cuda.synchronize()
            tol = 1e-13 if precision == pkg.FP64 else 1e-6
            assert rel_l2(yout.cpu().numpy(), ref.cpu().numpy()) < tol
        plan.check()
