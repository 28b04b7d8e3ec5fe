"""The library's host setup code (Sec. 2.1 knots and B-splines, Sec. 5
univariate factors, eq. eig_dec) checked on the CPU: tests/host_shim.cpp
exposes it through C entry points and is compiled here with g++ together with
the library's own host sources. References: NumPy's Gauss-Legendre rule and
SciPy's generalized symmetric eigensolver (library routines), and the oracle's
B-splines, knot elevation and univariate matrices (pinned in their own tests)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import splines, stokes, univariate as uv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1712_00403_gb300", "csrc")
D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ is not available")
    out = str(tmp_path_factory.mktemp("host_shim") / "libhostshim.so")
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", os.path.join(ROOT, "tests", "host_shim.cpp"),
           os.path.join(CSRC, "host_spline.cpp"), os.path.join(CSRC, "host_eig.cpp"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    i, d = ctypes.c_int, ctypes.c_double
    lib.shim_validate.argtypes = [D, i, i]
    lib.shim_elevate.argtypes = [D, i, D]
    lib.shim_gauss.argtypes = [i, D, D]
    lib.shim_eval.argtypes = [D, i, i, d, D, D]
    lib.shim_mixed.argtypes = [D, i, i, i, i, i, D, i, i, i, i, i, i, D]
    lib.shim_stiffness.argtypes = [D, i, i, i, i, i, d, d, i, D]
    lib.shim_gen_eig.argtypes = [D, D, i, D, D]
    return lib


def _p(a):
    return a.ctypes.data_as(D)


def _arr(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _space_args(s):
    """(knots, len, degree, first kept index, kept count) of an oracle space with contiguous indices."""
    assert np.array_equal(s.keep, np.arange(s.keep[0], s.keep[0] + s.n))
    t = _arr(s.knots)
    return t, len(t), s.degree, int(s.keep[0]), s.n


def test_knot_validation_and_elevation(shim):
    for n_el, p in ((1, 1), (5, 2), (7, 3), (4, 6)):
        t = _arr(synth.open_uniform_knots(n_el, p))
        assert shim.shim_validate(_p(t), len(t), p) == 1
        out = np.zeros(2 * len(t))
        m = shim.shim_elevate(_p(t), len(t), _p(out))
        np.testing.assert_array_equal(out[:m], splines.elevate_knots(t, p))
    # degree 1: one zero only, decreasing, not starting at 0, interior multiplicity 2 > p
    for bad in ([0, 0.5, 1, 1.0], [0, 0, 1, 1, 0.5], [0.1, 0.1, 1, 1.0], [0, 0, 0.5, 0.5, 1, 1]):
        t = _arr(bad)
        assert shim.shim_validate(_p(t), len(t), 1) == 0, bad


def test_gauss_legendre_matches_numpy(shim):
    for n in (1, 2, 3, 5, 8, 10):
        x, w = np.zeros(n), np.zeros(n)
        shim.shim_gauss(n, _p(x), _p(w))
        rx, rw = np.polynomial.legendre.leggauss(n)
        order = np.argsort(x)
        np.testing.assert_allclose(x[order], rx, atol=1e-15)
        np.testing.assert_allclose(w[order], rw, atol=1e-14)


def test_bspline_values_and_derivatives_match_oracle(shim):
    rng = np.random.default_rng(11)
    for t, p in ((synth.open_uniform_knots(6, 2), 2), (splines.elevate_knots(synth.open_uniform_knots(5, 3), 3), 4),
                 (splines.open_knots(4, 5, 2), 5)):
        t = _arr(t)
        xs = np.concatenate([rng.random(40), [0.0, 1.0, 0.5]])
        B, Dv = splines.basis(t, p, xs)
        N, dN = np.zeros(p + 1), np.zeros(p + 1)
        for q, x in enumerate(xs):
            s = shim.shim_eval(_p(t), len(t), p, float(x), _p(N), _p(dN))
            idx = np.arange(s - p, s + 1)
            full, dfull = np.zeros(B.shape[1]), np.zeros(B.shape[1])
            full[idx], dfull[idx] = N, dN
            np.testing.assert_allclose(full, B[q], atol=1e-14)
            np.testing.assert_allclose(dfull, Dv[q], atol=1e-11 * max(1.0, np.abs(Dv[q]).max()))


@pytest.mark.parametrize("disc", ["TH", "RT"])
def test_univariate_factors_match_oracle(shim, disc):
    """The factors of P_V and of the operator (Sec. 5): mass, stiffness (RT: with the
    Nitsche terms), and the mixed velocity/pressure products, at the p+2 point rule."""
    S = stokes.build([synth.open_uniform_knots(n, 3) for n in (5, 7, 4)], 3, disc)
    npts = S.p + 2
    for k in range(3):
        for d in range(3):
            sv = S.vel[k][d]
            t, nt, p, f, n = _space_args(sv)
            M = np.zeros((n, n))
            shim.shim_mixed(_p(t), nt, p, f, n, 0, _p(t), nt, p, f, n, 0, npts, _p(M))
            np.testing.assert_allclose(M, uv.mass(sv, npts=npts), atol=1e-15, rtol=1e-13)
            K = np.zeros((n, n))
            shim.shim_stiffness(_p(t), nt, p, f, n, int(sv.nitsche), sv.cpen, sv.h, npts, _p(K))
            np.testing.assert_allclose(K, uv.stiffness(sv, npts=npts), atol=1e-12 * np.abs(K).max())
            sp = S.pres[d]
            tq, ntq, pq, fq, nq = _space_args(sp)
            for da, db in ((0, 0), (0, 1), (1, 0)):
                X = np.zeros((nq, n))
                shim.shim_mixed(_p(tq), ntq, pq, fq, nq, da, _p(t), nt, p, f, n, db, npts, _p(X))
                ref = uv.mixed(sp, da, sv, db, npts=npts)
                np.testing.assert_allclose(X, ref, atol=1e-13 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("n_el", [6, 40])
def test_generalized_eigensolver(shim, n_el):
    """U^T M U = I, U^T K U = diag(lam) (eq. eig_dec) on the TH velocity pencil, and the
    eigenvalues against scipy.linalg.eigh(K, M). n_el = 6 runs the Jacobi branch
    (n <= 48), n_el = 40 the Householder + QL branch."""
    S = stokes.build([synth.open_uniform_knots(n_el, 2)], 2)
    sv = S.vel[0][0]
    M, K = uv.mass(sv), uv.stiffness(sv)
    n = M.shape[0]
    assert (n <= 48) == (n_el == 6)
    lam, U = np.zeros(n), np.zeros((n, n))
    assert shim.shim_gen_eig(_p(_arr(K)), _p(_arr(M)), n, _p(lam), _p(U)) == 1
    scale = np.abs(lam).max()
    np.testing.assert_allclose(U.T @ M @ U, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(U.T @ K @ U, np.diag(lam), atol=1e-12 * scale)
    np.testing.assert_allclose(np.sort(lam), scipy.linalg.eigh(K, M, eigvals_only=True), rtol=1e-11,
                               atol=1e-13 * scale)
    # a matrix that is not SPD is refused
    bad = _arr(M.copy())
    bad[0, 0] = -1.0
    assert shim.shim_gen_eig(_p(_arr(K)), _p(bad), n, _p(lam), _p(U)) == 0
