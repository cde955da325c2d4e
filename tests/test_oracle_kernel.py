"""Pins for the oracle's kernel (Eqs. 1-3) and its direct sum O_direct."""
import math

import numpy as np

from oracle.direct import direct_rows
from oracle.fdm import helmholtz, helmholtz_c


def test_closed_form_values():
    # r = 1/2, kappa = 2 pi: exp(i pi) / (4 pi / 2) = -1 / (2 pi)
    f = helmholtz(np.array([0.5, 0.0, 0.0]), np.zeros(3), 2 * math.pi)
    assert abs(f - (-1.0 / (2 * math.pi))) < 1e-15
    # r = 2, kappa = pi/4: exp(i pi/2) / (8 pi) = i / (8 pi)
    f = helmholtz(np.array([0.0, 2.0, 0.0]), np.zeros(3), math.pi / 4)
    assert abs(f - 1j / (8 * math.pi)) < 1e-16


def test_symmetry_modulus_and_zero_diagonal():
    rng = np.random.default_rng(0)
    x = rng.random((200, 3))
    y = rng.random((200, 3))
    f1 = helmholtz(x, y, 37.0)
    f2 = helmholtz(y, x, 37.0)
    assert np.array_equal(f1, f2)
    r = np.linalg.norm(x - y, axis=1)
    assert np.allclose(np.abs(f1), 1.0 / (4 * math.pi * r), rtol=1e-14)
    assert helmholtz(x[3], x[3], 5.0) == 0.0


def test_directional_rewrite_eq2():
    """f(x, y) = f_c(x, y) exp(i kappa <x, c>) exp(-i kappa <y, c>), Eqs. (2), (3)."""
    rng = np.random.default_rng(1)
    x = rng.random((50, 3))
    y = rng.random((50, 3)) + 2.0
    c = rng.standard_normal(3)
    c /= np.linalg.norm(c)
    kappa = 53.0
    lhs = helmholtz(x, y, kappa)
    rhs = helmholtz_c(x, y, kappa, c) * np.exp(1j * kappa * (x @ c)) * np.exp(-1j * kappa * (y @ c))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)


def test_direct_single_source_closed_form():
    tgt = np.array([[0.5, 0.0, 0.0], [0.0, 2.0, 0.0]])
    src = np.zeros((1, 3))
    x = np.array([2.0 - 1.0j])
    y = direct_rows(tgt, src, 2 * math.pi, x)
    assert abs(y[0] - x[0] * (-1.0 / (2 * math.pi))) < 1e-15
    y = direct_rows(tgt, src, math.pi / 4, x)
    assert abs(y[1] - x[0] * (1j / (8 * math.pi))) < 1e-15


def test_direct_linearity_rows_and_zero_diagonal():
    rng = np.random.default_rng(2)
    p = rng.random((300, 3))
    a = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    b = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    ya = direct_rows(p, p, 11.0, a)
    yb = direct_rows(p, p, 11.0, b)
    yab = direct_rows(p, p, 11.0, 2.0 * a - 3j * b)
    assert np.allclose(yab, 2.0 * ya - 3j * yb, rtol=1e-12, atol=1e-12)
    rows = np.array([299, 7, 0])
    assert np.array_equal(direct_rows(p, p, 11.0, a, rows), ya[rows])
    # zero diagonal: a unit vector on one source gives 0 at the same point
    e = np.zeros(300, dtype=complex)
    e[5] = 1.0
    assert direct_rows(p, p, 11.0, e, np.array([5]))[0] == 0.0
