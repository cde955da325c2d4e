"""FP64 CUDA path against the FP64 oracle: bit-exact trees and partition
tables, counters, and products within rel-l2 1e-10 (both sides FP64, the
difference is summation order and the box-centred phase form)."""
import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from oracle.direct import direct_rows
from oracle.fdm import FDMOracle
from paper_2004_14229_gb300.workloads import (complex_normal, sample_rows, tensor_grid,
                                              uniform_points, workload)
from tests.gpu_common import gpu_apply, morton_key, rel_l2

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _compare_trees(plan, oracle):
    for which, tree in ((0, oracle.tt), (1, oracle.ts)):
        assert plan.stats()["depth"] == tree.depth
        for lv in range(tree.depth + 1):
            keys, begin, end, perm = plan.export_tree(which, lv, with_perm=True)
            boxes = tree.by_level[lv]
            assert len(keys) == len(boxes)
            okeys = np.array([morton_key(tree.ijk[b], lv) for b in boxes], dtype=np.int64)
            assert np.array_equal(keys, okeys)
            for i, b in enumerate(boxes):
                got = perm[begin[i]:end[i]]
                if lv == tree.depth:          # a leaf keeps ascending original index
                    assert np.array_equal(got, tree.idx[b])
                else:                         # a larger box holds its children's runs in key order
                    assert np.array_equal(np.sort(got), tree.idx[b])


def _compare_offsets(plan, oracle):
    tt, ts = oracle.tt, oracle.ts
    bt = oracle.block_tree()
    want = {}
    for (t, s) in bt.adm:
        d = tuple(int(v) for v in (tt.ijk[t] - ts.ijk[s]))
        want.setdefault(t, set()).add((d, oracle.c_of_block(t, s)))
    for lv in range(1, tt.depth + 1):
        tables = [plan.export_offsets(lv, a) for a in range(8)]
        for t in tt.by_level[lv]:
            ijk = tt.ijk[t]
            alpha = int(ijk[0] & 1) + 2 * int(ijk[1] & 1) + 4 * int(ijk[2] & 1)
            off, dirs = tables[alpha]
            got = set()
            for d, c in zip(off, dirs):
                s_ijk = ijk - d
                if (lv,) + tuple(int(v) for v in s_ijk) in ts.key_to_box:
                    got.add((tuple(int(v) for v in d), int(c)))
            assert got == want.get(t, set()), (lv, t)
    st = plan.stats()
    bs = bt.stats(tt, ts)
    assert st["n_coupling"] == bs["N_C"]
    assert st["n_near_blocks"] == bs["near_blocks"]
    assert st["nf_entries"] == bs["nf_entries"]


def test_cfg1_small_workload_parity_tree_and_partition():
    t, s, x, w = workload("uniform-8k-k16-d4-o4")
    o = FDMOracle(t, s, w["kappa"], w["order"], [0, 0, 0], 1.0, w["depth"])
    with pkg.Plan(t, s, w["kappa"], order=w["order"], max_depth=w["depth"]) as plan:
        _compare_trees(plan, o)
        _compare_offsets(plan, o)
        y = gpu_apply(plan, x)
    yo = o.apply(x)
    assert rel_l2(y, yo) < TOL_FP64
    rows = sample_rows(t.shape[0], 512, 4)
    yd = direct_rows(t, s, w["kappa"], x, rows)
    # same approximation error as the oracle's (the method, not the arithmetic)
    assert abs(rel_l2(y[rows], yd) - rel_l2(yo[rows], yd)) < 1e-9


@pytest.mark.parametrize("nt,ns,kappa,order,depth,l_hf", [
    (1000, 777, 40.0, 3, 3, None),      # ragged sizes, l_hf = 3 (leaves high-frequency)
    (3000, 2500, 40.0, 4, 4, None),     # sub-face directions on level 3
    (2000, 2100, 12.0, 5, 3, 2),        # forced l_hf
    (1500, 1500, 9.0, 6, 3, -1),        # no high-frequency level
    (700, 900, 20.0, 2, 3, None),       # order 2
    (1200, 1100, 30.0, 7, 3, None),     # order 7
])
def test_fp64_parity_small_cases(nt, ns, kappa, order, depth, l_hf):
    t = uniform_points(nt, 11)
    s = uniform_points(ns, 12)
    x = complex_normal(ns, 13)
    o = FDMOracle(t, s, kappa, order, [0, 0, 0], 1.0, depth, l_hf=l_hf)
    with pkg.Plan(t, s, kappa, order=order, max_depth=depth, l_hf=l_hf) as plan:
        assert plan.stats()["l_hf"] == o.l_hf
        _compare_trees(plan, o)
        _compare_offsets(plan, o)
        y = gpu_apply(plan, x)
    assert rel_l2(y, o.apply(x)) < TOL_FP64


def test_paper_grid_k5_counts_and_parity():
    """Sect. 4 setup at k = 5 (P_S = P_T: coincident pairs give 0): the
    counters reproduce Table 1 and the product matches the oracle."""
    pts = tensor_grid(5)
    n = pts.shape[0]
    x = complex_normal(n, 3)
    with pkg.Plan(pts, pts, 3.2, order=5, max_depth=8, n_max=512,
                  root=((-1.0, -1.0, -1.0), 2.0)) as plan:
        st = plan.stats()
        assert (st["depth"], st["l_hf"]) == (2, 1)
        assert st["n_coupling"] == 3096 and st["n_stored_coupling"] == 316
        assert round(100.0 * st["nf_entries"] / n ** 2, 2) == 24.41
        y = gpu_apply(plan, x)
    rows = sample_rows(n, 64, 4)
    o = FDMOracle(pts, pts, 3.2, 5, [-1, -1, -1], 2.0, 8, n_max=512)
    assert rel_l2(y[rows], o.apply(x, rows=rows)) < TOL_FP64


def test_edge_cases_no_far_field_single_points_duplicates():
    # depth 1: every pair is nearfield, the product is the direct sum
    t = uniform_points(300, 1)
    s = uniform_points(200, 2)
    x = complex_normal(200, 3)
    with pkg.Plan(t, s, 5.0, order=3, max_depth=1) as plan:
        assert plan.stats()["n_coupling"] == 0
        assert rel_l2(gpu_apply(plan, x), direct_rows(t, s, 5.0, x)) < 1e-13
    # one target, one source: an admissible pair, so the far field approximates it
    t1 = np.array([[0.25, 0.5, 0.75]])
    s1 = np.array([[0.75, 0.5, 0.25]])
    x1 = np.array([1.0 - 2.0j])
    with pkg.Plan(t1, s1, 3.0, order=3, max_depth=3) as plan:
        assert plan.stats()["n_coupling"] == 1
        y = gpu_apply(plan, x1)
    o = FDMOracle(t1, s1, 3.0, 3, [0, 0, 0], 1.0, 3)
    assert rel_l2(y, o.apply(x1)) < TOL_FP64
    # P_T = P_S with duplicated points: coincident pairs contribute 0
    p = uniform_points(800, 5)
    p = np.concatenate([p, p[:100]])
    x = complex_normal(900, 6)
    o = FDMOracle(p, p, 18.0, 4, [0, 0, 0], 1.0, 3)
    with pkg.Plan(p, p, 18.0, order=4, max_depth=3) as plan:
        assert rel_l2(gpu_apply(plan, x), o.apply(x)) < TOL_FP64
    # points on box boundaries and on the root's lower faces
    b = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [1.0, 1.0, 1.0], [0.25, 0.75, 0.125],
                  [0.125, 0.0, 1.0]] * 3) + np.repeat(np.array([0.0, 0.0, 0.0])[None], 15, 0)
    b[5:10] *= 0.5
    x = complex_normal(15, 7)
    o = FDMOracle(b, b, 7.0, 3, [0, 0, 0], 1.0, 3)
    with pkg.Plan(b, b, 7.0, order=3, max_depth=3) as plan:
        _compare_trees(plan, o)
        assert rel_l2(gpu_apply(plan, x), o.apply(x)) < TOL_FP64


def test_apply_host_multi_rhs_and_errors():
    import torch
    t = uniform_points(2000, 1)
    s = uniform_points(1800, 2)
    xs = complex_normal(1800, 3, nrhs=3)
    with pkg.Plan(t, s, 20.0, order=4, max_depth=3, nrhs_max=3) as plan:
        y3 = gpu_apply(plan, xs)
        for r in range(3):
            assert rel_l2(y3[r], gpu_apply(plan, xs[r])) < 1e-15
        yh = plan.apply_host(xs)
        assert np.array_equal(yh, y3)
        with pytest.raises(pkg.DFDMError) as e:
            plan.apply(torch.zeros((4, 1800), dtype=torch.complex128, device="cuda"))
        assert e.value.status == 1
        plan.check()
