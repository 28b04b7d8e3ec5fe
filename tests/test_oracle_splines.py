"""Pins for oracle.splines (paper Sec. 2.1) against closed forms and invariants."""
from math import comb

import numpy as np
import pytest

from oracle import splines
import synth


@pytest.mark.parametrize("p,alpha,n_el", [(1, 0, 5), (2, 1, 7), (3, 2, 4), (4, 1, 3), (5, 4, 6), (3, 0, 3)])
def test_partition_of_unity_and_nonnegativity(p, alpha, n_el):
    t = splines.open_knots(n_el, p, alpha)
    x = np.concatenate([np.linspace(0, 1, 257), np.random.default_rng(0).random(100)])
    B, D = splines.basis(t, p, x)
    assert B.shape[1] == splines.dim(t, p)
    assert np.all(B >= -1e-15)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-11)


def test_dimension_formula():
    # m = p + 1 + (n_el - 1)(p - alpha); Taylor-Hood velocity (degree p+1, mult 2): 2 n_el + p
    for p in range(1, 7):
        for n_el in (1, 4, 16, 64):
            tq = splines.open_knots(n_el, p, p - 1)
            assert splines.dim(tq, p) == n_el + p
            tv = splines.elevate_knots(tq, p)
            assert splines.dim(tv, p + 1) == 2 * n_el + p
    # the configuration with 64^3 elements and p=3: 129 interior velocity functions per direction
    assert splines.dim(splines.elevate_knots(splines.open_knots(64, 3, 2), 3), 4) - 2 == 129


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_single_element_is_bernstein(p):
    t = np.array([0.0] * (p + 1) + [1.0] * (p + 1))
    x = np.linspace(0, 1, 33)
    B, D = splines.basis(t, p, x)
    for i in range(p + 1):
        bern = comb(p, i) * x ** i * (1 - x) ** (p - i)
        dbern = comb(p, i) * (i * x ** max(i - 1, 0) * (1 - x) ** (p - i) * (i > 0)
                              - (p - i) * x ** i * (1 - x) ** max(p - i - 1, 0) * (p - i > 0))
        np.testing.assert_allclose(B[:, i], bern, atol=1e-14)
        np.testing.assert_allclose(D[:, i], dbern, atol=1e-12)


def test_value_at_right_end():
    # reading: the last function equals 1 at eta = 1
    t = splines.open_knots(6, 3, 2)
    B, _ = splines.basis(t, 3, np.array([1.0, 0.0]))
    assert B[0, -1] == 1.0 and np.all(B[0, :-1] == 0.0)
    assert B[1, 0] == 1.0 and np.all(B[1, 1:] == 0.0)


@pytest.mark.parametrize("p,alpha,n_el", [(2, 1, 5), (3, 1, 4), (4, 3, 3)])
def test_integral_closed_form(p, alpha, n_el):
    t = splines.open_knots(n_el, p, alpha)
    x, w = splines.gauss_rule(t, p + 2)
    B, _ = splines.basis(t, p, x)
    ints = w @ B
    m = splines.dim(t, p)
    expect = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(m)])
    np.testing.assert_allclose(ints, expect, atol=1e-15)


def test_derivative_vs_finite_difference():
    rng = np.random.default_rng(3)
    inner = np.sort(rng.random(5))
    t = np.concatenate([[0] * 4, inner, inner[2:3], [1] * 4])   # non-uniform, one double knot
    t = np.sort(t)
    x = rng.random(40) * 0.98 + 0.01
    x = x[np.min(np.abs(x[:, None] - t[None, :]), axis=1) > 1e-4]
    h = 1e-6
    _, D = splines.basis(t, 3, x)
    Bp, _ = splines.basis(t, 3, x + h)
    Bm, _ = splines.basis(t, 3, x - h)
    np.testing.assert_allclose(D, (Bp - Bm) / (2 * h), atol=1e-5)


def test_gauss_rule_exactness():
    t = splines.open_knots(5, 2, 1)
    for npts in (1, 3, 6):
        x, w = splines.gauss_rule(t, npts)
        deg = 2 * npts - 1
        np.testing.assert_allclose(w @ x ** deg, 1.0 / (deg + 1), rtol=1e-14)


def test_synth_knots_match_definition():
    for p in (2, 3, 5):
        for n_el in (1, 3, 16):
            np.testing.assert_array_equal(synth.open_uniform_knots(n_el, p), splines.open_knots(n_el, p, p - 1))
