"""Pins for oracle.minres (Paige-Saunders MINRES, cited in paper Sec. 4)."""
import numpy as np
import pytest

from oracle import minres, stokes
import synth


def _sym_indef(rng, n):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([rng.uniform(1, 10, n // 2), -rng.uniform(1, 10, n - n // 2)])
    return Q @ np.diag(ev) @ Q.T


def test_vs_dense_solve_and_residual_estimate():
    rng = np.random.default_rng(0)
    n = 40
    A = _sym_indef(rng, n)
    L = rng.standard_normal((n, n))
    P = L @ L.T + n * np.eye(n)
    Pinv = np.linalg.inv(P)
    b = rng.standard_normal(n)
    hist = []
    x, info = minres.minres(lambda v: A @ v, b, lambda v: Pinv @ v, tol=1e-12, maxit=200, history=hist)
    assert info["status"] == "converged"
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:]))
    # |eta_j| is the P^{-1} norm of the residual at every step
    for j in (1, 5, 12):
        xj, _ = minres.minres(lambda v: A @ v, b, lambda v: Pinv @ v, tol=0.0, maxit=j)
        rj = b - A @ xj
        r0 = b
        est = hist[j]
        true = np.sqrt(rj @ Pinv @ rj) / np.sqrt(r0 @ Pinv @ r0)
        assert abs(est - true) < 1e-10


def test_ideal_block_preconditioner_three_iterations():
    rng = np.random.default_rng(4)
    n, m = 30, 12
    L = rng.standard_normal((n, n))
    A = L @ L.T + n * np.eye(n)
    B = rng.standard_normal((m, n))
    K = np.block([[A, B.T], [B, np.zeros((m, m))]])
    S = B @ np.linalg.solve(A, B.T)
    Pinv = np.block([[np.linalg.inv(A), np.zeros((n, m))], [np.zeros((m, n)), np.linalg.inv(S)]])
    b = rng.standard_normal(n + m)
    x, info = minres.minres(lambda v: K @ v, b, lambda v: Pinv @ v, tol=1e-10, maxit=50)
    assert info["status"] == "converged" and info["iters"] <= 3
    np.testing.assert_allclose(K @ x, b, atol=1e-8)


def test_stokes_pd_minres_small():
    """P_D-MINRES on the 2D Taylor-Hood system: converges, the true residual is
    small and the constant-pressure component stays out of the iterate."""
    S = stokes.build_uniform(6, 2, 2)
    A = stokes.assembled(S)
    b = synth.rhs(1, S.block_sizes)
    x, info = minres.minres(lambda v: A @ v, b, lambda v: stokes.apply_PD_inv(S, v), tol=1e-10, maxit=300)
    assert info["status"] == "converged"
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-8
    # iterates lie in P^{-1} range(A): the pressure block satisfies 1^T P_Q p = 0
    from oracle import kron
    PQ = kron.kron_matrix(stokes.pq_factors(S))
    pr = x[-S.block_sizes[-1]:]
    assert abs(np.ones(len(pr)) @ PQ @ pr) < 1e-9 * np.linalg.norm(pr)


def test_true_residual_check_reaches_tolerance():
    """With true_check the returned iterate meets ||b - A x||_2 <= tol ||b||_2
    (the estimate-only rule can stop above it)."""
    S = stokes.build_uniform(8, 2, 2)
    A = stokes.assembled(S)
    b = synth.rhs(3, S.block_sizes)
    Pinv = lambda v: stokes.apply_PD_inv(S, v)
    x1, i1 = minres.minres(lambda v: A @ v, b, Pinv, tol=1e-8, maxit=500)
    x2, i2 = minres.minres(lambda v: A @ v, b, Pinv, tol=1e-8, maxit=500, true_check=True)
    assert i2["iters"] >= i1["iters"]
    assert np.linalg.norm(b - A @ x2) / np.linalg.norm(b) <= 1e-8
