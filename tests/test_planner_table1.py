"""The library's planner (csrc/planner.cu, host code) against Table 1 of
Sect. 4, all five printed rows k = 5..9: on the tensor grid with n_max = 512
every box of the depth-(k-3) uniform tree is occupied, so N_C, N_SC and the
nearfield share follow from the planner's per-level offset tables alone
(dfdm_uniform_counts, no points, no GPU).  The oracle's own block tree pins
k = 5..7 in test_oracle_blocktree.py; k = 8, 9 (1.7e7 and 1.3e8 points) are
checked only here."""
import json
import os

import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg

TABLE = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1.json")))


@pytest.mark.parametrize("k", [5, 6, 7, 8, 9])
def test_table1_counts_from_the_planner(k):
    row = TABLE["rows"][str(k)]
    # root [-1, 1]^3 (side 2), depth k - 3, kappa = 0.1 2^k, eta2 = 5, l_hf = k - 4
    nc, nsc, near = pkg.uniform_counts(row["kappa"], k - 3, eta2=5.0, root_side=2.0, l_hf=k - 4)
    assert nc == row["N_C"]
    assert nsc == row["N_SC"]
    leaf_points = 512
    nf = 100.0 * near * leaf_points ** 2 / float(row["N"]) ** 2
    digits = len(str(row["nf_percent"]).split(".")[1])
    assert round(nf, digits) == pytest.approx(row["nf_percent"]), nf
    # the default high-frequency rule gives the same partition (reading R12: l_hf = k - 4)
    assert pkg.uniform_counts(row["kappa"], k - 3, eta2=5.0, root_side=2.0) == (nc, nsc, near)


def test_uniform_counts_rejects_bad_arguments():
    for args in ((0.0, 3), (1.0, -1), (1.0, 11)):
        with pytest.raises(pkg.DFDMError) as e:
            pkg.uniform_counts(*args)
        assert e.value.status == 1


@pytest.mark.parametrize("k,depth,kappa", [(4, 3, 6.0), (4, 3, 40.0), (4, 4, 8.0)])
def test_offset_tables_match_the_oracle_block_tree(k, depth, kappa):
    """Every (offset, direction) the planner lists for a target box of the
    fully occupied grid is an admissible block of the oracle's Alg. 2 with
    the direction of Def. 3, and nothing is missing (bit-exact)."""
    from oracle.fdm import FDMOracle
    from paper_2004_14229_gb300.workloads import tensor_grid
    pts = tensor_grid(k)                     # 8^k points: every box down to depth k occupied
    o = FDMOracle(pts, pts, kappa, 2, [-1.0, -1.0, -1.0], 2.0, depth)
    tt, ts = o.tt, o.ts
    assert all(len(tt.by_level[lv]) == 8 ** lv for lv in range(depth + 1))
    want = {}
    for (t, s) in o.block_tree().adm:
        d = tuple(int(v) for v in (tt.ijk[t] - ts.ijk[s]))
        want.setdefault(t, set()).add((d, o.c_of_block(t, s)))
    for lv in range(1, depth + 1):
        tables = [pkg.uniform_offsets(kappa, depth, lv, a, root_side=2.0, l_hf=o.l_hf) for a in range(8)]
        for t in tt.by_level[lv]:
            ijk = tt.ijk[t]
            alpha = int(ijk[0] & 1) + 2 * int(ijk[1] & 1) + 4 * int(ijk[2] & 1)
            off, dirs = tables[alpha]
            got = set()
            g = 1 << lv
            for d, c in zip(off, dirs):
                s_ijk = ijk - d
                if all(0 <= v < g for v in s_ijk):
                    got.add((tuple(int(v) for v in d), int(c)))
            assert got == want.get(t, set()), (lv, t)


@pytest.mark.parametrize("k", [6, 7, 8])
def test_direction_indices_within_the_direction_sets(k):
    """Alg. 3: level l <= l_hf has 6 4^(l_hf - l) directions, coarser levels
    none (index 0); every coupling offset's direction index is in range and
    the finest high-frequency level uses all six faces."""
    kappa, depth, lhf = 0.1 * 2 ** k, k - 3, k - 4
    for lv in range(1, depth + 1):
        used = set()
        for a in range(8):
            _, dirs = pkg.uniform_offsets(kappa, depth, lv, a, root_side=2.0, l_hf=lhf)
            used.update(int(c) for c in dirs)
        if not used:              # no admissible block on this level (the coarsest ones)
            continue
        if lv <= lhf:
            assert max(used) < 6 * 4 ** (lhf - lv) and min(used) >= 0, lv
        else:
            assert used == {0}, lv
        if lv == lhf:
            assert used == set(range(6))


def _adm(d, level, kappa, eta2, side):
    """(A1) and (A3) of Def. 1 for boxes of `level` at integer offset d, by the oracle."""
    from oracle.fdm import admissibility
    w = side / 2 ** level
    lo_t = [0.0, 0.0, 0.0]
    hi_t = [w, w, w]
    lo_s = [-d[i] * w for i in range(3)]
    hi_s = [lo_s[i] + w for i in range(3)]
    a1, a3 = admissibility(lo_t, hi_t, lo_s, hi_s, kappa, eta2)
    return a1 and a3


def test_offsets_are_alg2_leaves_for_random_parameters():
    """For random kappa, eta2, root side and depth: every listed offset d is
    admissible on its level (Def. 1 by the oracle) and its parent pair, whose
    offset is ceil((d - alpha) / 2), is not -- the leaves of Alg. 2 -- and
    the counts agree with the tables."""
    rng = np.random.default_rng(17)
    for _ in range(12):
        kappa = float(np.exp(rng.uniform(np.log(1.0), np.log(60.0))))
        eta2 = float(rng.choice([2.0, 5.0, 8.0]))
        side = float(rng.choice([1.0, 2.0]))
        depth = int(rng.integers(2, 5))
        for lv in range(1, depth + 1):
            for alpha in range(8):
                off, _ = pkg.uniform_offsets(kappa, depth, lv, alpha, eta2=eta2, root_side=side)
                al = [(alpha >> i) & 1 for i in range(3)]
                if len(off) > 40:                    # a random sample keeps the test short
                    off = off[rng.choice(len(off), 40, replace=False)]
                for d in off:
                    assert _adm(d, lv, kappa, eta2, side), (kappa, eta2, side, lv, tuple(d))
                    dp = [-((al[i] - int(d[i])) // 2) for i in range(3)]
                    assert not _adm(dp, lv - 1, kappa, eta2, side), (kappa, eta2, side, lv, tuple(d))
