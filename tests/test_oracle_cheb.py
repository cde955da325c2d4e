"""Pins for the oracle's Chebyshev interpolation (Eq. 4 with reading R1) and the
transfer matrices (Eq. 13, Sect. 2.7)."""
import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as P

from oracle.fdm import box_lagrange, box_nodes, cheb_nodes, lagrange_1d


def test_nodes_are_chebyshev_roots():
    for order in range(2, 11):
        r = np.sort(cheb_nodes(order))
        roots = np.sort(C.chebroots([0] * order + [1]))
        assert np.allclose(r, roots, atol=1e-14)
        assert np.all(np.diff(cheb_nodes(order)) < 0)   # nu ascending, coordinate descending


def test_lagrange_cardinal_and_partition_of_unity():
    for order in (3, 5, 7):
        r = cheb_nodes(order)
        assert np.allclose(lagrange_1d(order, r), np.eye(order), atol=1e-13)
        t = np.linspace(-1, 1, 101)
        assert np.allclose(lagrange_1d(order, t).sum(axis=1), 1.0, atol=1e-13)


def test_interpolation_exact_for_degree_m_tensor_polynomials():
    rng = np.random.default_rng(5)
    for order in (3, 4, 6):
        m = order - 1
        cx, cy, cz = (rng.standard_normal(m + 1) for _ in range(3))
        lo = np.array([0.25, -1.0, 3.0])
        hi = lo + 0.125

        def poly(p):
            return P.polyval(p[:, 0], cx) * P.polyval(p[:, 1], cy) * P.polyval(p[:, 2], cz)

        xi = box_nodes(lo, hi, order)
        pts = lo + (hi - lo) * rng.random((40, 3))
        approx = box_lagrange(lo, hi, order, pts) @ poly(xi)
        assert np.allclose(approx, poly(pts), rtol=1e-11, atol=1e-11)
        # the multi-index order: node k = nu_x + o nu_y + o^2 nu_z
        r = cheb_nodes(order)
        mid, half = (lo + hi) / 2, (hi - lo) / 2
        k = 1 + order * 2 + order * order * (order - 1)
        assert np.allclose(xi[k], mid + half * np.array([r[1], r[2], r[order - 1]]))


def test_transfer_reference_matrix_is_exact_on_polynomials():
    """E_{t'}[j, k] = L_{t,k}(xi_{t',j}) maps parent nodal values of a degree-m
    polynomial to its child nodal values exactly, for all 8 octants."""
    rng = np.random.default_rng(6)
    order = 5
    m = order - 1
    coef = rng.standard_normal((3, m + 1))
    lo, hi = np.zeros(3), np.ones(3)

    def poly(p):
        return np.prod([P.polyval(p[:, i], coef[i]) for i in range(3)], axis=0)

    xi_par = box_nodes(lo, hi, order)
    for q in range(8):
        bits = np.array([q & 1, (q >> 1) & 1, (q >> 2) & 1])
        clo = lo + 0.5 * bits
        xi_ch = box_nodes(clo, clo + 0.5, order)
        e = box_lagrange(lo, hi, order, xi_ch)
        assert np.allclose(e @ poly(xi_par), poly(xi_ch), rtol=1e-12, atol=1e-12)
