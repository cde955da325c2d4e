"""Pins for the oracle's admissibility (Def. 1) and block tree (Alg. 2, Def. 2):
Table 1 of Sect. 4 reproduced exactly, plus brute-force structure checks."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle.fdm import BlockTree, ClusterTree, admissibility, default_l_hf
from paper_2004_14229_gb300.workloads import tensor_grid

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))


def _paper_setup(k):
    pts = tensor_grid(k)
    tree = ClusterTree(pts, [-1, -1, -1], 2.0, 512, 64)
    kappa = 0.1 * 2 ** k
    return tree, kappa


@pytest.mark.parametrize("k", [5, 6, pytest.param(7, marks=pytest.mark.slow)])
def test_table1_counts_exact(k):
    tree, kappa = _paper_setup(k)
    bt = BlockTree(tree, tree, kappa, 5.0)
    st = bt.stats(tree, tree)
    row = GOLDEN["rows"][str(k)]
    assert st["N_C"] == row["N_C"]
    assert st["N_SC"] == row["N_SC"]
    # the table prints nf% rounded to two (k=5..7) significant decimals
    digits = len(str(row["nf_percent"]).split(".")[1])
    assert round(st["nf_percent"], digits) == row["nf_percent"]


@pytest.mark.parametrize("k", [5, 6])
def test_paper_side_facts(k):
    """Sect. 4: depth k-3 = l_hf + 1, all inadmissible blocks on that level,
    at most 27 nearfield blocks per leaf; l_hf = k - 4 by reading R12."""
    tree, kappa = _paper_setup(k)
    assert default_l_hf(kappa, 2.0, tree.depth) == k - 4
    bt = BlockTree(tree, tree, kappa, 5.0)
    per_leaf = {}
    for (t, s) in bt.near:
        assert tree.level[t] == k - 3
        per_leaf[t] = per_leaf.get(t, 0) + 1
    assert max(per_leaf.values()) == 27


def test_admissibility_against_brute_force_distance():
    rng = np.random.default_rng(3)
    w = 0.125
    for _ in range(300):
        a = rng.integers(0, 8, 3)
        b = rng.integers(0, 8, 3)
        lo_t, hi_t = a * w, a * w + w
        lo_s, hi_s = b * w, b * w + w
        g = np.linspace(0, 1, 9)
        grid = np.array(list(itertools.product(g, g, g)))
        pt = lo_t + w * grid
        ps = lo_s + w * grid
        dist = math.sqrt(np.min(np.sum((pt[:, None, :] - ps[None, :, :]) ** 2, axis=-1)))
        diam = math.sqrt(3) * w
        for kappa, eta2 in ((20.0, 5.0), (3.0, 1.5)):
            a1, a3 = admissibility(lo_t, hi_t, lo_s, hi_s, kappa, eta2)
            assert a1 == (diam <= eta2 * dist + 1e-12)
            assert a3 == (kappa * diam ** 2 <= eta2 * dist + 1e-12)


def test_block_tree_partitions_the_matrix():
    """Def. 2: the leaves t^ x s^ tile {1..N_T} x {1..N_S} exactly once."""
    rng = np.random.default_rng(4)
    tp = rng.random((300, 3))
    sp = rng.random((250, 3))
    tt = ClusterTree(tp, [0, 0, 0], 1.0, 3, 6)
    ts = ClusterTree(sp, [0, 0, 0], 1.0, 3, 6)
    bt = BlockTree(tt, ts, 9.0, 5.0)
    cover = np.zeros((300, 250), dtype=np.int64)
    for (t, s) in bt.adm + bt.near:
        cover[np.ix_(tt.idx[t], ts.idx[s])] += 1
    assert np.all(cover == 1)
    for (t, s) in bt.adm:
        assert all(admissibility(tt.lo[t], tt.hi[t], ts.lo[s], ts.hi[s], 9.0, 5.0))
        assert tt.level[t] == ts.level[s]
    for (t, s) in bt.near:
        assert not all(admissibility(tt.lo[t], tt.hi[t], ts.lo[s], ts.hi[s], 9.0, 5.0))
        assert tt.is_leaf[t] or ts.is_leaf[s]
