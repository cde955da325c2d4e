"""Host-side pieces of bench.py and of the selector's data (no GPU): the
profile summaries it cites parse, the M2L traffic figure is tied to the M2L
kernel's source, and the selector labels follow their stated rule."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fp64_comparator_summary_parses():
    c = bench._fp64_comparator("uniform-4M-k128-d7-o6")
    assert c["s_per_product"] > 0 and c["value"] == pytest.approx(1.0 / c["s_per_product"])
    assert c["rel_err_vs_oracle_rows"] < 1e-10
    assert bench._fp64_comparator("no-such-workload") is None


def test_traffic_follows_the_m2l_source(tmp_path, monkeypatch):
    t = bench._traffic("uniform-4M-k128-d7-o6")
    assert t is not None and t > 1e11
    # a copy of the tree whose M2L section differs: the figure is withdrawn
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2004_14229_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "m2l_pair_uniform-4M-k128-d7-o6_dram.md"), root / "profiles")
    csrc = os.path.join(ROOT, "paper_2004_14229_gb300", "csrc")
    shutil.copy(os.path.join(csrc, "sm100_ptx.cuh"), root / "paper_2004_14229_gb300" / "csrc")
    text = open(os.path.join(csrc, "tc.cu")).read()
    (root / "paper_2004_14229_gb300" / "csrc" / "tc.cu").write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic("uniform-4M-k128-d7-o6") == t
    # a change outside the M2L section keeps it
    (root / "paper_2004_14229_gb300" / "csrc" / "tc.cu").write_text(text + "\n// trailing comment\n")
    assert bench._traffic("uniform-4M-k128-d7-o6") == t
    # a change inside it does not
    marker = "struct M2lArgs {"
    (root / "paper_2004_14229_gb300" / "csrc" / "tc.cu").write_text(text.replace(marker, marker + " ", 1))
    assert bench._traffic("uniform-4M-k128-d7-o6") is None


def _rec(errs, orders, lhf=3, errs_m1=None):
    err = {(o, 0): e for o, e in zip(orders, errs)}
    for o, e in zip(orders, errs_m1 or []):
        err[(o, -1)] = e
    return dict(kappa=10.0, n=4000, depth=3, root_side=1.0, l_hf=lhf, err=err, orders=tuple(orders))


ERRS = [1e-1, 3e-2, 3e-3, 5e-4, 6e-5, 7e-6]   # orders 2..7


def test_selector_labels():
    from paper_2004_14229_gb300 import selector_data as D
    o = (2, 3, 4, 5, 6, 7)
    r = _rec(ERRS, o)
    # the smallest order within tol / 3
    assert D.labels(r, 1e-2)[0] == 4          # 3e-3 <= 3.3e-3
    assert D.labels(r, 3e-3)[0] == 5          # 5e-4 <= 1e-3
    assert D.labels(r, 1e-6)[0] == 8          # none: one above the highest measured
    # a record measured in the tensor-core form only (orders 2..6)
    rt = _rec(ERRS[:5], o[:5])
    assert D.labels(rt, 1e-5)[0] == 7
    # l_hf - 1 is taken when it still meets tol / 3 at the chosen order
    rl = _rec(ERRS, o, errs_m1=[1e-1, 3e-2, 2e-3, 5e-4, 6e-5, 7e-6])
    assert D.labels(rl, 1e-2) == (4, 2)
    rl2 = _rec(ERRS, o, errs_m1=[1e-1, 3e-2, 9e-3, 5e-4, 6e-5, 7e-6])
    assert D.labels(rl2, 1e-2) == (4, 3)


def test_selector_samples_have_one_row_per_level_and_tolerance():
    from paper_2004_14229_gb300._build import build_library
    from paper_2004_14229_gb300 import selector_data as D
    build_library()                          # the features come from the library (host code)
    o = (2, 3, 4, 5, 6, 7)
    recs = [_rec(ERRS, o), dict(_rec([1e-1] * 5, o[:5]), depth=4)]
    X, T = D.make_samples(recs, [1e-2, 1e-4])
    assert X.shape == (2 * 2 + 2 * 3, 4) and T.shape == (10, 2)
    assert T[0, 0] == pytest.approx((4 - 2) / 8.0)             # first record, tol 1e-2
    assert T[-1, 0] == pytest.approx((7 - 2) / 8.0)            # second record: none suffices


def test_selector_record_json_round_trip():
    import json
    r = _rec(ERRS, (2, 3, 4, 5, 6, 7), errs_m1=[1e-1, 3e-2, 2e-3, 5e-4, 6e-5, 7e-6])
    j = json.loads(json.dumps(bench.selector_record_json(r)))
    assert j["orders"] == [2, 3, 4, 5, 6, 7] and j["l_hf"] == 3
    back = {(o, sh): e for o, sh, e in j["err"]}
    assert back == r["err"]
