"""dfdm_direct_rows_noalloc: the direct-sum rows for callers that cannot
allocate device memory (their device memory belongs to another framework's
caching allocator, or they run a loop that must not let an allocation call
stall the device).  The call writes its partial sums to the library's fixed
device scratch instead of allocating; this test checks, through the C ABI,
that two calls in a row give what dfdm_direct_rows gives, and that a request
larger than the fixed scratch is refused.  The file is collected last."""
import ctypes

import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from paper_2004_14229_gb300.workloads import complex_normal, sample_rows, uniform_points
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the tolerance of the direct-sum tests


def _case(nt, ns, nrows, seed):
    import torch
    t = torch.from_numpy(uniform_points(nt, seed)).cuda()
    s = torch.from_numpy(uniform_points(ns, seed + 1)).cuda()
    x = torch.from_numpy(complex_normal(ns, seed + 2)).cuda()
    rows = torch.from_numpy(sample_rows(nt, nrows, seed + 3)).cuda()
    return t, s, x, rows


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    lib = pkg.load_library()
    for nt, ns, nrows, kappa, seed in ((30000, 25000, 4096, 23.0, 100), (5000, 70000, 777, 51.0, 200)):
        t, s, x, rows = _case(nt, ns, nrows, seed)
        ref = pkg.direct_rows(t, s, kappa, x, rows)
        y = torch.full((nrows,), float("nan"), dtype=torch.complex128, device="cuda")
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        status = lib.dfdm_direct_rows_noalloc(ctypes.c_void_p(t.data_ptr()), nt, ctypes.c_void_p(s.data_ptr()), ns,
                                              kappa, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(rows.data_ptr()),
                                              nrows, ctypes.c_void_p(y.data_ptr()), st)
        assert status == 0, lib.dfdm_last_error()
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), ref.cpu().numpy()) < TOL


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    lib = pkg.load_library()
    nrows = (1 << 18) + 1
    t, s, x, _ = _case(1000, 1000, 10, 300)
    rows = torch.zeros(nrows, dtype=torch.int64, device="cuda")
    y = torch.zeros(nrows, dtype=torch.complex128, device="cuda")
    status = lib.dfdm_direct_rows_noalloc(ctypes.c_void_p(t.data_ptr()), 1000, ctypes.c_void_p(s.data_ptr()), 1000,
                                          5.0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(rows.data_ptr()),
                                          nrows, ctypes.c_void_p(y.data_ptr()), None)
    assert status == 1
    assert b"262144" in lib.dfdm_last_error()
    assert int(torch.count_nonzero(y).item()) == 0
