"""Pins of the ACA oracle (oracle/aca.py, Sect. 2.7 closing remark) against
facts that do not come from it: an exactly rank-r matrix is recovered with
rank r; a full-rank matrix is reproduced after n steps; the zero matrix has
rank 0; on a smooth kernel between separated clusters the error meets the
tolerance and the rank stays near the SVD's numerical rank (numpy's SVD, an
independent routine); and in Alg. 4 the ACA mode converges to the
uncompressed product as the tolerance goes to 0."""
import numpy as np
import pytest

from oracle.aca import aca_partial
from oracle.fdm import FDMOracle, cheb_nodes
from paper_2004_14229_gb300.workloads import complex_normal


def _rel_fro(a, u, v):
    return np.linalg.norm(a - u @ v.conj().T) / np.linalg.norm(a)


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("r", [1, 3, 7])
def test_exact_low_rank_is_recovered(r):
    rng = np.random.default_rng(r)
    a = _cplx(rng, 60, r) @ _cplx(rng, r, 45)
    u, v = aca_partial(a, 1e-13)
    # r terms, plus at most the rounding-level term that meets the stop test
    assert u.shape[1] in (r, r + 1) and v.shape == (45, u.shape[1])
    if u.shape[1] == r + 1:
        assert np.linalg.norm(u[:, r]) * np.linalg.norm(v[:, r]) <= 1e-13 * np.linalg.norm(a)
    assert _rel_fro(a, u[:, :r], v[:, :r]) < 1e-12


def test_full_rank_matrix_after_n_steps():
    rng = np.random.default_rng(5)
    a = _cplx(rng, 20, 20)
    u, v = aca_partial(a, 0.0)
    assert u.shape[1] == 20
    assert _rel_fro(a, u, v) < 1e-10


def test_zero_and_single_entry():
    u, v = aca_partial(np.zeros((7, 5)), 1e-8)
    assert u.shape == (7, 0) and v.shape == (5, 0)
    a = np.zeros((7, 5), dtype=complex)
    a[4, 2] = 2.0 - 1.0j                      # row 0 is zero: the next rows are tried
    u, v = aca_partial(a, 1e-12)
    assert u.shape[1] == 1 and _rel_fro(a, u, v) == 0.0


def test_max_rank_caps_the_rank():
    rng = np.random.default_rng(6)
    a = _cplx(rng, 30, 30)
    u, v = aca_partial(a, 1e-12, max_rank=4)
    assert u.shape[1] == 4


def _grid(order, lo):
    g = (cheb_nodes(order) + 1.0) / 2.0            # nodes in [0, 1]
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) + np.asarray(lo)


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_smooth_kernel_meets_tolerance_near_svd_rank(tol):
    """Helmholtz kernel between two unit boxes whose centres are 3 apart
    (an admissible pair at low frequency), on order-6 tensor Chebyshev grids:
    n = 216, the situation of a coupling matrix."""
    xt = _grid(6, [0.0, 0.0, 0.0])
    ys = _grid(6, [3.0, 0.0, 0.0])
    kappa = 2.0
    d = np.linalg.norm(xt[:, None, :] - ys[None, :, :], axis=2)
    a = np.exp(1j * kappa * d) / (4.0 * np.pi * d)
    u, v = aca_partial(a, tol)
    err = _rel_fro(a, u, v)
    sv = np.linalg.svd(a, compute_uv=False)
    # numerical rank at the same relative Frobenius accuracy
    tail = np.sqrt(np.cumsum((sv ** 2)[::-1]))[::-1] / np.linalg.norm(sv)
    k_svd = int(np.count_nonzero(tail > tol))
    assert err < 20 * tol
    assert k_svd <= u.shape[1] <= 2 * k_svd + 4
    assert u.shape[1] < 216 // 2


def test_alg4_with_aca_converges_to_uncompressed():
    rng = np.random.default_rng(7)
    t = rng.random((900, 3))
    s = rng.random((850, 3))
    x = complex_normal(850, 8)
    o = FDMOracle(t, s, 12.0, 4, [0, 0, 0], 1.0, 3)
    y = o.apply(x, mode="reuse")
    errs = []
    for tol in (1e-3, 1e-6, 1e-10):
        ya = o.apply(x, mode="aca", aca_tol=tol)
        errs.append(np.linalg.norm(ya - y) / np.linalg.norm(y))
        ranks = list(o.last_aca_ranks.values())
        assert ranks and max(ranks) <= 64
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9
    assert errs[0] < 1e-2
