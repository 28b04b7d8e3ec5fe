"""Pins for oracle.kron (paper Sec. 2.3 identities, eq. eig_dec, Algorithm 1)."""
import numpy as np
import pytest

from oracle import kron, stokes, splines, univariate as uv


def _rand_spd(rng, n):
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


@pytest.mark.parametrize("shape", [(3, 4), (2, 3, 4), (5, 1, 3)])
def test_mode_products_vs_explicit_kron(shape):
    rng = np.random.default_rng(1)
    dims = shape                                   # (n1, n2[, n3])
    factors = [rng.standard_normal((d + 1, d)) for d in dims]    # rectangular too
    x = rng.standard_normal(int(np.prod(dims)))
    np.testing.assert_allclose(kron.kron_apply(factors, x), kron.kron_matrix(factors) @ x, atol=1e-12)
    # vec index i = i1 + (i2-1) n1 + ... : a unit vector e_(i1,i2,...) maps to column of the Kronecker matrix
    e = np.zeros(len(x)); e[1] = 1.0            # i1 = 2, others 1
    col = kron.kron_matrix(factors)[:, 1]
    np.testing.assert_allclose(kron.kron_apply(factors, e), col, atol=0)


def test_generalized_eig_identities():
    t = splines.elevate_knots(splines.open_knots(16, 3, 2), 3)
    s = uv.interior_space(t, 4)
    K, M = uv.stiffness(s), uv.mass(s)
    lam, U = kron.gen_eig(K, M)
    np.testing.assert_allclose(U.T @ M @ U, np.eye(len(lam)), atol=1e-12)
    np.testing.assert_allclose(U.T @ K @ U, np.diag(lam), atol=1e-12 * lam.max())
    assert np.all(lam > 0)


@pytest.mark.parametrize("dims,coef", [((5, 7), (2.0, 1.0)), ((4, 3, 5), (1.0, 2.0, 1.0)), ((3, 4, 4), (1.0, 1.0, 1.0))])
def test_fd_equals_dense_lu_random(dims, coef):
    rng = np.random.default_rng(7)
    Ks = [_rand_spd(rng, n) for n in dims]
    Ms = [_rand_spd(rng, n) for n in dims]
    t = rng.standard_normal(int(np.prod(dims)))
    q_fd = kron.fd_solve(Ks, Ms, coef, t)
    q_lu = kron.dense_solve(Ks, Ms, coef, t)
    np.testing.assert_allclose(q_fd, q_lu, rtol=0, atol=1e-12 * np.abs(q_lu).max())
    # residual of eq. sylv_eq
    np.testing.assert_allclose(kron.kron_sum_apply(Ks, Ms, coef, q_fd), t, atol=1e-10)


@pytest.mark.parametrize("dim,p,n_el", [(2, 2, 3), (3, 2, 2), (3, 3, 2), (2, 4, 2)])
def test_fd_equals_dense_lu_spline_pencils(dim, p, n_el):
    S = stokes.build_uniform(n_el, p, dim)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(S.n_total)
    s_fd = stokes.apply_PD_inv(S, r, "fd")
    s_lu = stokes.apply_PD_inv(S, r, "dense")
    rel = np.linalg.norm(s_fd - s_lu) / np.linalg.norm(s_lu)
    assert rel < 1e-12


def test_mass_solve_banded_vs_dense():
    rng = np.random.default_rng(5)
    Ms = [uv.mass(uv.full_space(splines.open_knots(n, p, p - 1), p)) for n, p in ((4, 2), (3, 3), (5, 1))]
    t = rng.standard_normal(int(np.prod([M.shape[0] for M in Ms])))
    np.testing.assert_allclose(kron.kron_mass_solve(Ms, t), np.linalg.solve(kron.kron_matrix(Ms), t),
                               rtol=1e-10, atol=1e-10)
