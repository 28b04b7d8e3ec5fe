"""Pins for oracle.univariate (paper Sec. 5 univariate factors) against closed forms."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import splines, univariate as uv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cardinal_stencils.txt")


def _stencils():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out[(int(f[0]), f[1])] = np.array([float(Fraction(v)) for v in f[2:]])
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_cardinal_stencils(p):
    n_el = 12
    h = 1.0 / n_el
    t = splines.open_knots(n_el, p, p - 1)
    s = uv.full_space(t, p)
    M, K = uv.mass(s), uv.stiffness(s)
    st = _stencils()
    mid = splines.dim(t, p) // 2          # a row far from both boundaries
    np.testing.assert_allclose(M[mid, mid - p:mid + p + 1], h * st[(p, "mass")], rtol=1e-13)
    if (p, "stiff") in st:
        np.testing.assert_allclose(K[mid, mid - p:mid + p + 1], st[(p, "stiff")] / h, rtol=1e-12)
    # band structure: functions overlap iff |i-j| <= p
    i, j = np.nonzero(np.abs(M) > 0)
    assert np.max(np.abs(i - j)) == p


@pytest.mark.parametrize("p,alpha", [(2, 1), (4, 3), (3, 1), (4, 2)])
def test_row_sums_before_removal(p, alpha):
    t = splines.open_knots(7, p, alpha)
    s = uv.full_space(t, p)
    M, K = uv.mass(s), uv.stiffness(s)
    m = splines.dim(t, p)
    np.testing.assert_allclose(M.sum(axis=1), [(t[i + p + 1] - t[i]) / (p + 1) for i in range(m)], atol=1e-15)
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-10 * np.abs(K).max())
    np.testing.assert_allclose(M, M.T, atol=0)
    np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())


def test_dirichlet_removal_and_spd():
    t = splines.elevate_knots(splines.open_knots(8, 3, 2), 3)
    s = uv.interior_space(t, 4)
    assert s.n == splines.dim(t, 4) - 2
    full = uv.full_space(t, 4)
    np.testing.assert_allclose(uv.mass(s), uv.mass(full)[1:-1, 1:-1], atol=0)
    assert np.all(np.linalg.eigvalsh(uv.stiffness(s)) > 0)
    assert np.all(np.linalg.eigvalsh(uv.mass(s)) > 0)


def test_exactness_vs_higher_order_rule():
    t = splines.elevate_knots(splines.open_knots(5, 3, 2), 3)
    s = uv.interior_space(t, 4)
    for fn in (uv.mass, uv.stiffness):
        np.testing.assert_allclose(fn(s, npts=5), fn(s, npts=9), rtol=0, atol=1e-14 * np.abs(fn(s)).max())


def test_derivative_mass_integration_by_parts():
    # int b_i' b_j + int b_i b_j' = [b_i b_j]_0^1 ; zero on the interior space
    t = splines.elevate_knots(splines.open_knots(6, 2, 1), 2)
    full, inner = uv.full_space(t, 3), uv.interior_space(t, 3)
    C = uv.mixed(full, 1, full, 0)
    B = np.zeros_like(C)
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(C + C.T, B, atol=1e-13)
    Ci = uv.mixed(inner, 1, inner, 0)
    np.testing.assert_allclose(Ci + Ci.T, 0.0, atol=1e-13)


def _coeffs(s, f):
    """Coefficients of f in the full spline space by L2 projection (exact for f in the space)."""
    x, w = splines.gauss_rule(s.knots, s.degree + 4)
    B, _ = splines.basis(s.knots, s.degree, x)
    return np.linalg.solve(uv.mass(s, npts=s.degree + 4), B.T @ (w * f(x)))


def test_nitsche_stiffness_closed_form():
    """cf^T K~ cg for polynomials f, g against the closed-form Nitsche bilinear
    form int f'g' - [f'(1)g(1) - f'(0)g(0) + g'(1)f(1) - g'(0)f(0)] + 2 C/h (f(1)g(1) + f(0)g(0))."""
    p, n_el, C = 3, 5, 15.0
    t = splines.open_knots(n_el, p, p - 1)
    s = uv.full_space(t, p, nitsche=True, cpen=C, h=1.0 / n_el)
    f = lambda x: 1 + 2 * x - x ** 3
    g = lambda x: 3 * x ** 2 - 0.5 * x + 0.25
    fp = lambda x: 2 - 3 * x ** 2
    gp = lambda x: 6 * x - 0.5
    cf, cg = _coeffs(s, f), _coeffs(s, g)
    # int_0^1 f' g' by exact polynomial integration
    P = np.polynomial.Polynomial
    integ = (P([2, 0, -3]) * P([-0.5, 6])).integ()
    vol = integ(1) - integ(0)
    expect = (vol - (fp(1) * g(1) - fp(0) * g(0) + gp(1) * f(1) - gp(0) * f(0))
              + 2 * C * n_el * (f(1) * g(1) + f(0) * g(0)))
    assert abs(cf @ uv.stiffness(s) @ cg - expect) < 1e-10 * abs(expect)
    K = uv.stiffness(s)
    np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    assert np.all(np.linalg.eigvalsh(K) > 0)
