"""The measured launch-shape tuner (dfdm_plan_autotune): the tuned product
equals the untuned one up to the rounding order of sums, the choice is one of
the timed candidates, and the JSON-lines cache gives it back without timing."""
import json

import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from paper_2004_14229_gb300.workloads import complex_normal, tensor_grid, uniform_points
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def _cases():
    t = tensor_grid(5)
    yield "grid-k5", t, t, 3.2, dict(order=5, max_depth=8, n_max=512, root=((-1.0, -1.0, -1.0), 2.0))
    yield "uniform-d5", uniform_points(200000, 51), uniform_points(200000, 52), 48.0, dict(order=5, max_depth=5)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_autotune_choice_cache_and_result(case, tmp_path):
    import torch
    name, t, s, kappa, kw = case
    x = torch.from_numpy(complex_normal(s.shape[0], 53).astype(np.complex64)).cuda()
    cache = str(tmp_path / "tune.jsonl")
    with pkg.Plan(t, s, kappa, precision=pkg.TC_FP16X3, **kw) as plan:
        y0 = plan.apply(x).cpu().numpy()
        tu = plan.autotune(x, cache=cache)
        plan.check()
        y1 = plan.apply(x).cpu().numpy()
        plan.check()
        st = plan.stats()
    print(name, tu)
    assert not tu["from_cache"] and tu["products"] >= 4
    assert 0 < tu["tuned_ms"] <= tu["rule_ms"]
    assert rel_l2(y1, y0) < 1e-6
    for lv in range(st["depth"] + 1):
        if st["level_coupling"][lv] > 0:
            assert tu["m2l_nsplit"][lv] > 0, lv
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["m2l_nsplit"] == tu["m2l_nsplit"] and rec["p2p"] == [tu["p2p_threads"], tu["p2p_chunks"]]
    # a new plan of the same shape takes the cached choice without timing
    with pkg.Plan(t, s, kappa, precision=pkg.TC_FP16X3, **kw) as plan:
        tc = plan.autotune(x, cache=cache)
        y2 = plan.apply(x).cpu().numpy()
        plan.check()
    assert tc["from_cache"] and tc["products"] == 0
    assert tc["m2l_nsplit"] == tu["m2l_nsplit"] and tc["p2p_threads"] == tu["p2p_threads"]
    assert rel_l2(y2, y0) < 1e-6
    assert len(open(cache).read().splitlines()) == 1


def test_autotune_rejects_fp64_plans_and_foreign_cache_lines(tmp_path):
    import torch
    t = uniform_points(20000, 54)
    x = torch.from_numpy(complex_normal(20000, 55).astype(np.complex64)).cuda()
    with pkg.Plan(t, t, 8.0, order=4, max_depth=3, precision=pkg.FP64) as plan:
        with pytest.raises(pkg.DFDMError) as e:
            plan.autotune(x)
        assert e.value.status == 1
    cache = tmp_path / "tune.jsonl"
    with pkg.Plan(t, t, 8.0, order=4, max_depth=3, precision=pkg.TC_FP16X3) as plan:
        plan.autotune(x, cache=str(cache))
        rec = json.loads(cache.read_text().splitlines()[0])
    rec["m2l_nsplit"] = [63] * 16                  # not a shape this plan would time
    cache.write_text(json.dumps(rec) + "\n")
    with pkg.Plan(t, t, 8.0, order=4, max_depth=3, precision=pkg.TC_FP16X3) as plan:
        with pytest.raises(pkg.DFDMError) as e:
            plan.autotune(x, cache=str(cache))
        assert e.value.status == 1
