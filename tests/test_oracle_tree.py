"""Pins for the oracle's uniform box cluster tree (Alg. 1, readings R3-R5) by
brute force over the points."""
import numpy as np
import pytest

from oracle.fdm import ClusterTree


def _check_tree(tree, pts, n_max, max_depth):
    n = pts.shape[0]
    seen = np.zeros(n, dtype=np.int64)
    for b in tree.leaves:
        idx = tree.idx[b]
        seen[idx] += 1
        assert np.all(np.diff(idx) > 0)                       # ascending index set
        lo, hi = tree.lo[b], tree.hi[b]
        p = pts[idx]
        on_closed_lower_face = (p == tree.root_lo) & (lo == tree.root_lo)
        assert np.all(((p > lo) | on_closed_lower_face) & (p <= hi))
        assert idx.size <= n_max or tree.level[b] == max_depth
    assert np.all(seen == 1)                                   # every point in exactly one leaf
    for b in range(tree.nboxes):
        w = tree.root_side / 2 ** tree.level[b]
        assert np.allclose(tree.hi[b] - tree.lo[b], w, rtol=0, atol=0)   # identical up to translation
        assert np.array_equal(tree.lo[b], tree.root_lo + w * tree.ijk[b])
        assert tree.idx[b].size >= 1                           # no empty boxes
        ch = tree.children[b]
        if ch:
            assert tree.idx[b].size > n_max
            assert np.array_equal(np.sort(np.concatenate([tree.idx[c] for c in ch])), tree.idx[b])
            octs = [int(np.dot(tree.ijk[c] - 2 * tree.ijk[b], [1, 2, 4])) for c in ch]
            assert octs == sorted(octs) and all(0 <= q < 8 for q in octs)
            for c in ch:
                assert tree.parent[c] == b and tree.level[c] == tree.level[b] + 1


@pytest.mark.parametrize("n_max,max_depth", [(0, 3), (10, 6), (1, 5)])
def test_tree_brute_force_uniform(n_max, max_depth):
    pts = np.random.default_rng(7).random((700, 3))
    tree = ClusterTree(pts, [0, 0, 0], 1.0, n_max, max_depth)
    _check_tree(tree, pts, n_max, max_depth)
    if n_max == 0:
        assert all(tree.level[b] == max_depth for b in tree.leaves)


def test_tree_boundaries_go_to_lower_box_and_closed_root_faces():
    pts = np.array([[0.5, 0.5, 0.5], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0],
                    [0.25, 0.75, 0.5], [0.5000000000000001, 0.5, 0.0]])
    tree = ClusterTree(pts, [0, 0, 0], 1.0, 0, 2)
    _check_tree(tree, pts, 0, 2)
    leaf_of = tree.leaf_of_point()
    assert tuple(tree.ijk[leaf_of[0]]) == (1, 1, 1)       # x = centre -> lower halves
    assert tuple(tree.ijk[leaf_of[1]]) == (0, 0, 0)       # root lower corner
    assert tuple(tree.ijk[leaf_of[2]]) == (3, 3, 3)
    assert tuple(tree.ijk[leaf_of[3]]) == (0, 2, 1)
    assert tuple(tree.ijk[leaf_of[4]]) == (2, 1, 0)


def test_tree_levels_are_morton_ordered_and_paper_grid_depth():
    from paper_2004_14229_gb300.workloads import tensor_grid
    for k in (4, 5):
        pts = tensor_grid(k)
        tree = ClusterTree(pts, [-1, -1, -1], 2.0, 512, 30)
        assert tree.depth == k - 3                              # Sect. 4: depth k - 3
        assert all(tree.idx[b].size == 512 for b in tree.leaves)
        for lv in range(tree.depth + 1):
            keys = []
            for b in tree.by_level[lv]:
                i = tree.ijk[b]
                key = 0
                for bit in range(lv):
                    key |= ((int(i[0]) >> bit) & 1) << (3 * bit)
                    key |= ((int(i[1]) >> bit) & 1) << (3 * bit + 1)
                    key |= ((int(i[2]) >> bit) & 1) << (3 * bit + 2)
                keys.append(key)
            assert keys == sorted(keys)


def test_tree_rejects_bad_points():
    with pytest.raises(ValueError):
        ClusterTree(np.array([[0.5, 0.5, 1.5]]), [0, 0, 0], 1.0, 0, 2)
    with pytest.raises(ValueError):
        ClusterTree(np.array([[0.5, np.nan, 0.5]]), [0, 0, 0], 1.0, 0, 2)
