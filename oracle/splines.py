"""Univariate B-splines and quadrature (paper Sec. 2.1). Oracle: test infrastructure only.

Pins (tests/test_oracle_splines.py): partition of unity and nonnegativity,
the single-element case equals the Bernstein basis, the closed form
int b_i = (xi_{i+p+1} - xi_i)/(p+1), derivative vs. a finite difference of
the values, exactness of the (p+2)-point Gauss rule vs. a higher-order rule.
"""
import numpy as np


def open_knots(n_el, degree, regularity):
    """Open uniform knot vector (Sec. 2.1): degree+1 copies of 0 and of 1,
    interior breakpoints j/n_el each repeated (degree - regularity) times
    (continuity + multiplicity = degree at a breakpoint)."""
    mult = degree - regularity
    if not (1 <= mult <= degree + 1):
        raise ValueError("regularity must lie in [-1, degree-1]")
    inner = np.repeat(np.arange(1, n_el, dtype=np.float64) / n_el, mult)
    return np.concatenate([np.zeros(degree + 1), inner, np.ones(degree + 1)])


def elevate_knots(knots, degree):
    """Knot vector of the space of degree+1 with the same regularity at every
    breakpoint (Taylor-Hood velocity, Sec. 2.2.1): each breakpoint's
    multiplicity grows by one."""
    z, counts = np.unique(knots, return_counts=True)
    return np.repeat(z, counts + 1).astype(np.float64)


def dim(knots, degree):
    """m = number of B-splines of the knot vector."""
    return len(knots) - degree - 1


def breakpoints(knots):
    return np.unique(knots)


def basis(knots, degree, x):
    """All B-splines of the knot vector and their first derivatives at x.

    Cox-de Boor recursion (Sec. 2.1) from piecewise constants with 0/0 = 0.
    The last nonzero span is closed on the right so that b_m(1) = 1
    (reading: the half-open degree-0 indicator would give 0 at eta = 1).
    Derivative: b_i^p' = p b_i^{p-1}/(xi_{i+p}-xi_i) - p b_{i+1}^{p-1}/(xi_{i+p+1}-xi_{i+1}).
    Returns (B, D) with shape (len(x), m).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = np.asarray(knots, dtype=np.float64)
    nint = len(t) - 1
    last = max(i for i in range(nint) if t[i] < t[i + 1])
    b = np.zeros((len(x), nint))
    for i in range(nint):
        if t[i] < t[i + 1]:
            inside = (t[i] <= x) & (x < t[i + 1])
            if i == last:
                inside |= x == t[i + 1]
            b[:, i] = inside
    prev = b
    for p in range(1, degree + 1):
        cur = np.zeros((len(x), nint - p))
        for i in range(nint - p):
            d1 = t[i + p] - t[i]
            d2 = t[i + p + 1] - t[i + 1]
            if d1 > 0:
                cur[:, i] += (x - t[i]) / d1 * prev[:, i]
            if d2 > 0:
                cur[:, i] += (t[i + p + 1] - x) / d2 * prev[:, i + 1]
        if p == degree:
            der = np.zeros_like(cur)
            for i in range(nint - p):
                d1 = t[i + p] - t[i]
                d2 = t[i + p + 1] - t[i + 1]
                if d1 > 0:
                    der[:, i] += p / d1 * prev[:, i]
                if d2 > 0:
                    der[:, i] -= p / d2 * prev[:, i + 1]
            return cur, der
        prev = cur
    # degree 0
    return prev, np.zeros_like(prev)


def gauss_rule(knots, npts):
    """Gauss-Legendre rule with npts points on every nonzero knot span.
    Reading: the paper is silent; the configurations use p+2 points per
    element (p = pressure degree), exact for all parametric M and K."""
    g, w = np.polynomial.legendre.leggauss(npts)
    z = breakpoints(knots)
    xs, ws = [], []
    for a, b in zip(z[:-1], z[1:]):
        xs.append(0.5 * (b - a) * g + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(xs), np.concatenate(ws)
