"""Univariate Galerkin matrices (paper Sec. 5, eq. prec3D_TH / prec3D_RT and the
univariate factors below them; Appendix for the weighted ones).
Oracle: test infrastructure only.

A univariate space is a knot vector, a degree, the list of kept basis indices
(Dirichlet removal drops the first and last function) and an optional
Nitsche boundary treatment (the RT tangential factors K~). Every matrix is
int_0^1 w(eta) b_i^(da)(eta) b_j^(db)(eta) deta by Gauss quadrature on the
common breakpoints, restricted to the kept indices.

Pins (tests/test_oracle_univariate.py): textbook cardinal B-spline stencils
(degree 1 and 2), M 1 = (xi_{i+p+1}-xi_i)/(p+1) before removal, K 1 = 0
before removal, symmetry, exactness vs. a higher-order rule, Nitsche terms
against a direct evaluation of the boundary values.
"""
from dataclasses import dataclass, field

import numpy as np

from . import splines


@dataclass
class Space1D:
    knots: np.ndarray
    degree: int
    keep: np.ndarray            # kept basis indices (0-based)
    nitsche: bool = False       # add the Nitsche boundary terms to the stiffness (K~)
    cpen: float = 0.0           # penalty constant C_pen
    h: float = 1.0              # mesh size in the penalty C_pen / h

    @property
    def n(self):
        return len(self.keep)

    @property
    def m(self):
        return splines.dim(self.knots, self.degree)


def interior_space(knots, degree):
    """Dirichlet removal: indices 2..m-1 (1-based) are kept."""
    m = splines.dim(knots, degree)
    return Space1D(np.asarray(knots, float), degree, np.arange(1, m - 1))


def full_space(knots, degree, nitsche=False, cpen=0.0, h=1.0):
    m = splines.dim(knots, degree)
    return Space1D(np.asarray(knots, float), degree, np.arange(m), nitsche, cpen, h)


def _rule(sa, sb, npts):
    knots = np.union1d(sa.knots, sb.knots)
    return splines.gauss_rule(knots, npts)


def default_npts(sa, sb):
    # p+2 points per element for the Taylor-Hood pair (p = pressure degree,
    # velocity degree p+1); in general enough points for exact polynomial products.
    return (sa.degree + sb.degree) // 2 + 1


def mixed(sa, da, sb, db, weight=None, npts=None):
    """[X]_{ij} = int_0^1 w b_{a,i}^(da) b_{b,j}^(db) over kept indices."""
    if npts is None:
        npts = default_npts(sa, sb)
    x, w = _rule(sa, sb, npts)
    if weight is not None:
        w = w * weight(x)
    Ba, Da = splines.basis(sa.knots, sa.degree, x)
    Bb, Db = splines.basis(sb.knots, sb.degree, x)
    Fa = (Ba, Da)[da][:, sa.keep]
    Fb = (Bb, Db)[db][:, sb.keep]
    return Fa.T @ (w[:, None] * Fb)


def mass(s, weight=None, npts=None):
    return mixed(s, 0, s, 0, weight, npts)


def stiffness(s, weight=None, npts=None, tau0=1.0, tau1=1.0):
    """int w b' b'; for a Nitsche space the tangential RT factor K~ (Sec. 5):
    minus [b_l'(1)b_s(1) - b_l'(0)b_s(0) + b_s'(1)b_l(1) - b_s'(0)b_l(0)
           - 2 C_pen/h (b_l(1)b_s(1) + b_l(0)b_s(0))],
    with the boundary values scaled by tau(0), tau(1) in the weighted case (Appendix)."""
    K = mixed(s, 1, s, 1, weight, npts)
    if s.nitsche:
        K = K - nitsche_boundary(s, tau0, tau1)
    return K


def nitsche_boundary(s, tau0=1.0, tau1=1.0):
    """The bracket subtracted from int tau b'b' in K~ (Sec. 5; Appendix for the
    weights): tau(1) b_l'(1) b_s(1) - tau(0) b_l'(0) b_s(0) + (l <-> s)
    - 2 C_pen/h (tau(1) b_l(1) b_s(1) + tau(0) b_l(0) b_s(0))."""
    B, D = splines.basis(s.knots, s.degree, np.array([0.0, 1.0]))
    b0, b1 = B[0, s.keep], B[1, s.keep]
    d0, d1 = D[0, s.keep], D[1, s.keep]
    return (tau1 * np.outer(d1, b1) - tau0 * np.outer(d0, b0)
            + tau1 * np.outer(b1, d1) - tau0 * np.outer(b0, d0)
            - 2.0 * s.cpen / s.h * (tau1 * np.outer(b1, b1) + tau0 * np.outer(b0, b0)))
