"""Pins for the oracle's directions: Alg. 3 (D^(l)), Def. 3 (dir_(l)) and the
(A2) cone condition they are built to satisfy."""
import itertools
import math

import numpy as np
import pytest

from oracle.fdm import Directions, default_l_hf


def _interleave(iu, iv, r):
    j = 0
    for b in range(r):
        j |= ((iv >> b) & 1) << (2 * b)
        j |= ((iu >> b) & 1) << (2 * b + 1)
    return j


def _face_index_integer(d, r):
    """j(v) of Def. 3 for an integer vector, from the geometry of the ray alone:
    first axis attaining max |v_i| (closed faces, smallest index wins), its sign,
    then the sub-face cell along u and v with boundary ties to the lower cell."""
    m = max(abs(int(x)) for x in d)
    axis = next(i for i in range(3) if abs(int(d[i])) == m)
    f = 2 * axis + (1 if d[axis] > 0 else 0)
    u, v = [a for a in range(3) if a != axis]

    def cell(x):
        num = (int(x) + m) * 2 ** r
        den = 2 * m
        return max(0, -(-num // den) - 1)          # ceil(num/den) - 1, clamped
    return f * 4 ** r + _interleave(cell(d[u]), cell(d[v]), r)


@pytest.mark.parametrize("l_hf", [0, 1, 3])
def test_counts_norms_and_self_map(l_hf):
    dirs = Directions(l_hf, l_hf + 2)
    for lv in range(0, l_hf + 1):
        assert dirs.count(lv) == 6 * 4 ** (l_hf - lv)          # Sect. 3, #D^(l)
        assert np.allclose(np.linalg.norm(dirs.vectors[lv], axis=1), 1.0)
        for j in range(dirs.count(lv)):
            assert dirs.dir(lv, dirs.vector(lv, j)) == j
            if lv < l_hf:                                     # E^(l)_{4(j-1)+1..4j} subdivide E^(l+1)_j
                assert dirs.dir(lv + 1, dirs.vector(lv, j)) == j // 4
    for lv in range(l_hf + 1, l_hf + 3):
        assert dirs.count(lv) == 1 and dirs.dir(lv, [1.0, 2.0, 3.0]) == 0


def test_dir_map_matches_ray_geometry_on_integer_offsets():
    l_hf = 3
    dirs = Directions(l_hf, l_hf)
    for lv in range(0, l_hf + 1):
        r = l_hf - lv
        for d in itertools.product(range(-7, 8), repeat=3):
            if d == (0, 0, 0):
                continue
            assert dirs.dir(lv, np.array(d, dtype=float) * 0.0625) == _face_index_integer(d, r)


def test_dir_map_random_rays_and_cone_condition_a2():
    """(A2): every ray lies in the cone of its sub-face, so |u - c| <= sqrt(2) 2^-r."""
    rng = np.random.default_rng(9)
    l_hf = 4
    dirs = Directions(l_hf, l_hf)
    v = rng.standard_normal((2000, 3))
    for lv in range(0, l_hf + 1):
        r = l_hf - lv
        for x in v:
            j = dirs.dir(lv, x)
            u = x / np.linalg.norm(x)
            assert np.linalg.norm(u - dirs.vector(lv, j)) <= math.sqrt(2) * 2.0 ** (-r) + 1e-12
            m = np.max(np.abs(x))
            axis = int(np.argmax(np.abs(x)))
            f = 2 * axis + (1 if x[axis] > 0 else 0)
            a, b = [i for i in range(3) if i != axis]
            cu = min(int(math.floor((x[a] / m + 1) * 2 ** (r - 1))), 2 ** r - 1)
            cv = min(int(math.floor((x[b] / m + 1) * 2 ** (r - 1))), 2 ** r - 1)
            assert j == f * 4 ** r + _interleave(cu, cv, r)


@pytest.mark.parametrize("k", [5, 6, 7, 8, 9])
def test_l_hf_rule_gives_paper_choice(k):
    assert default_l_hf(0.1 * 2 ** k, 2.0, k - 3) == k - 4
