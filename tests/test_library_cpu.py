"""Host-side checks of the C ABI library (no GPU needed): it loads, exports every
symbol include/dfdm.h declares, and its host-only calls behave."""
import ctypes
import os
import re

import pytest

import paper_2004_14229_gb300 as pkg

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dfdm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2004_14229_gb300._build import build_library
    build_library()
    return pkg.load_library()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(dfdm_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(pkg.EXPORTED_SYMBOLS) == sorted(names)


def test_params_default_and_version(lib):
    p = pkg.Params()
    assert lib.dfdm_params_default(ctypes.byref(p)) == 0
    assert (p.order, p.max_depth, p.n_max, p.eta2, p.l_hf) == (5, 6, 0, 5.0, -2)
    assert p.root_side == 1.0 and p.nrhs_max == 1
    assert lib.dfdm_params_default(None) == 1
    assert b"sm_103a" in lib.dfdm_version()
    assert lib.dfdm_last_error()


def test_invalid_arguments_return_status(lib):
    import numpy as np
    pts = np.random.default_rng(0).random((10, 3))
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Plan(pts, pts, -1.0)
    assert e.value.status == 1
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Plan(pts, pts, 1.0, order=11)
    assert e.value.status == 1
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Plan(bad, pts, 1.0)
    assert e.value.status == 1
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Plan(pts + 2.0, pts, 1.0)          # outside the unit root cube
    assert e.value.status == 1
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Plan(pts, pts, 1.0, order=7, precision=pkg.TC_FP16X3)   # tensor-core form: orders 2..6
    assert e.value.status == 6
    assert lib.dfdm_plan_destroy(None) == 0
    assert lib.dfdm_apply(None, None, None, 1, None) == 1
    assert lib.dfdm_plan_autotune(None, None, None, None, None) == 1


def test_plan_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    pts = np.random.default_rng(0).random((10, 3))
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Plan(pts, pts, 1.0, max_depth=2)
    assert e.value.status in (2, 3)


def test_batch_invalid_arguments(lib):
    import ctypes
    import numpy as np
    pts = np.random.default_rng(0).random((10, 3))
    prob = [dict(targets=pts, sources=pts, kappa=1.0)]
    with pytest.raises(pkg.DFDMError) as e:
        pkg.Batch([], order=3)
    assert e.value.status == 1
    p = pkg.Params()
    assert lib.dfdm_params_default(ctypes.byref(p)) == 0
    p.n_max = 8                                 # batches use uniform trees
    arr = (pkg.Problem * 1)()
    arr[0].targets, arr[0].n_t = pts.ctypes.data, 10
    arr[0].sources, arr[0].n_s = pts.ctypes.data, 10
    arr[0].kappa, arr[0].max_depth = 1.0, -1
    out = ctypes.c_void_p(0)
    assert lib.dfdm_batch_create(1, arr, ctypes.byref(p), 0, None, ctypes.byref(out)) == 1
    p.n_max = 0
    assert lib.dfdm_batch_create(1, arr, ctypes.byref(p), 65, None, ctypes.byref(out)) == 1
    assert lib.dfdm_batch_destroy(None) == 0
    assert lib.dfdm_batch_apply(None, None, None, 1, None) == 1
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        with pytest.raises(pkg.DFDMError) as e:
            pkg.Batch(prob, order=3, max_depth=1, root=((0, 0, 0), 1.0))
        assert e.value.status in (2, 3)


def test_selector_features_and_argument_checks(lib):
    import ctypes
    import numpy as np
    assert lib.dfdm_selector_param_count() == 8770
    # the four features of include/dfdm.h, written out
    kappa, side, level, n, tol = 40.0, 2.0, 3, 100000, 1e-5
    f = pkg.Selector.features(kappa, side, level, n, tol)
    w = side / 2 ** level
    want = [level / 10, np.log2(kappa * np.sqrt(3) * w) / 8, np.log2(1 + n / 8 ** level) / 16, 5 / 10]
    assert np.allclose(f, want, rtol=1e-6)
    out = np.empty(4, dtype=np.float32)
    for bad in ((0.0, 1.0, 2, 10, 1e-3), (1.0, -1.0, 2, 10, 1e-3), (1.0, 1.0, -1, 10, 1e-3),
                (1.0, 1.0, 2, 0, 1e-3), (1.0, 1.0, 2, 10, 0.0)):
        assert lib.dfdm_selector_features(*bad, out.ctypes.data) == 1
    th = np.zeros(8770, dtype=np.float32)
    x = np.zeros(4, dtype=np.float32)
    y = np.zeros(2, dtype=np.float32)
    assert lib.dfdm_selector_forward(None, x.ctypes.data, 1, y.ctypes.data, None) == 1
    assert lib.dfdm_selector_forward(th.ctypes.data, x.ctypes.data, 0, y.ctypes.data, None) == 1
    assert lib.dfdm_selector_train(th.ctypes.data, x.ctypes.data, y.ctypes.data, 1, 5, ctypes.c_float(0.0),
                                   th.ctypes.data, None, None) == 1
    p = pkg.Params()
    assert lib.dfdm_params_default(ctypes.byref(p)) == 0
    p.max_depth = 11
    assert lib.dfdm_select_params(th.ctypes.data, 10.0, 1e-4, 1000, ctypes.byref(p), None) == 1
    with pytest.raises(ValueError):
        pkg.Selector(np.zeros(10, dtype=np.float32))
