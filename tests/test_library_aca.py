"""The library's host-side ACA (dfdm_aca, Sect. 2.7) against the oracle's
(oracle/aca.py): the same steps give the same rank and the same factors to
rounding, on exactly low-rank matrices and on the Helmholtz kernel between
separated Chebyshev grids; argument checks.  No GPU."""
import ctypes

import numpy as np
import pytest

import paper_2004_14229_gb300 as pkg
from oracle.aca import aca_partial


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2004_14229_gb300._build import build_library
    build_library()


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _grid(order, lo):
    from oracle.fdm import cheb_nodes
    g = (cheb_nodes(order) + 1.0) / 2.0
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) + np.asarray(lo)


def _cases():
    rng = np.random.default_rng(11)
    yield "rank5", _cplx(rng, 60, 5) @ _cplx(rng, 5, 45), 1e-13
    xt, ys = _grid(6, [0.0, 0.0, 0.0]), _grid(6, [2.5, 1.0, 0.0])
    d = np.linalg.norm(xt[:, None, :] - ys[None, :, :], axis=2)
    a = np.exp(1j * 4.0 * d) / (4.0 * np.pi * d)
    yield "helmholtz-1e-4", a, 1e-4
    yield "helmholtz-1e-8", a, 1e-8
    yield "random", _cplx(rng, 17, 23), 0.0


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_library_aca_equals_oracle(case):
    _, a, tol = case
    u, v = pkg.aca(a, tol)
    uo, vo = aca_partial(a, tol)
    assert u.shape == uo.shape and v.shape == vo.shape
    scale = np.linalg.norm(a)
    assert np.linalg.norm(u @ v.conj().T - uo @ vo.conj().T) <= 1e-12 * scale
    # term by term (late terms are small, so compare them on the matrix's scale)
    for l in range(u.shape[1]):
        t, to = np.outer(u[:, l], v[:, l].conj()), np.outer(uo[:, l], vo[:, l].conj())
        assert np.linalg.norm(t - to) <= 1e-10 * scale


def test_library_aca_caps_and_checks():
    rng = np.random.default_rng(12)
    a = _cplx(rng, 30, 30)
    u, v = pkg.aca(a, 0.0, max_rank=4)
    assert u.shape == (30, 4) and v.shape == (30, 4)
    u, v = pkg.aca(np.zeros((6, 9)), 1e-6)
    assert u.shape == (6, 0) and v.shape == (9, 0)
    lib = pkg.load_library()
    k = ctypes.c_int(0)
    buf = np.zeros(64, dtype=np.complex128)
    assert lib.dfdm_aca(None, 4, 4, 1e-6, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(k)) == 1
    assert lib.dfdm_aca(buf.ctypes.data, 0, 4, 1e-6, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(k)) == 1
    assert lib.dfdm_aca(buf.ctypes.data, 4, 4, -1.0, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(k)) == 1
    assert lib.dfdm_aca(buf.ctypes.data, 4, 4, 1e-6, 4, None, None, ctypes.byref(k)) == 1
    assert lib.dfdm_aca(buf.ctypes.data, 4, 4, 1e-6, 0, None, None, ctypes.byref(k)) == 0 and k.value == 0
