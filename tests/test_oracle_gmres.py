"""Pins for oracle.gmres and the block triangular / constraint preconditioners
of oracle.stokes (paper Sec. 4, eq. P_T, eq. P_C and the product form of
P_C^{-1})."""
import numpy as np
import pytest

from oracle import gmres, kron, minres, stokes


def test_gmres_solves_random_nonsymmetric_systems():
    rng = np.random.default_rng(5)
    for n in (5, 12, 30):
        A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.3
        M = np.diag(rng.uniform(0.5, 2.0, n))
        b = rng.standard_normal(n)
        x, info = gmres.gmres(lambda v: A @ v, b, lambda v: np.linalg.solve(M, v), tol=1e-12, maxit=n)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)
        assert info["status"] == "converged" and info["iters"] <= n


def test_gmres_estimate_is_the_preconditioned_residual_and_never_increases():
    rng = np.random.default_rng(6)
    n = 25
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    Mi = np.diag(1.0 / rng.uniform(1.0, 3.0, n))
    b = rng.standard_normal(n)
    hist = []
    for k in range(1, 8):
        hist.clear()
        x, info = gmres.gmres(lambda v: A @ v, b, lambda v: Mi @ v, tol=0.0, maxit=k, history=hist)
        direct = np.linalg.norm(Mi @ (b - A @ x)) / np.linalg.norm(Mi @ b)
        assert abs(hist[-1] - direct) <= 1e-12 * max(1.0, direct)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-14) for i in range(len(hist) - 1))


def _ideal_blocks(dim, n_el):
    S = stokes.build_uniform(n_el, 2, dim)
    A = stokes.assembled(S)
    d = S.dim
    off = np.concatenate([[0], np.cumsum(S.block_sizes)])
    Av = A[:off[d], :off[d]]
    Bt = A[:off[d], off[d]:]
    Sch = Bt.T @ np.linalg.solve(Av, Bt)
    return S, A, Av, Bt, Sch, off[d]


def test_ideal_block_triangular_converges_in_two_steps():
    """P_T = [[A, B^T], [0, -S]], S = B A^{-1} B^T: (P^{-1} 𝒜 - I)^2 = 0 on the
    complement of the constant pressure, so GMRES stops after 2 steps."""
    S, A, Av, Bt, Sch, nv = _ideal_blocks(2, 3)
    P = np.zeros_like(A)
    P[:nv, :nv] = Av
    P[:nv, nv:] = Bt
    P[nv:, nv:] = -(Sch + np.ones_like(Sch) / Sch.shape[0])   # + 11^T/n: S is singular on constants
    rng = np.random.default_rng(7)
    b = A @ rng.standard_normal(A.shape[0])                    # consistent right-hand side
    x, info = gmres.gmres(lambda v: A @ v, b, lambda v: np.linalg.solve(P, v), tol=1e-10, maxit=10)
    assert info["status"] == "converged" and info["iters"] == 2


def test_ideal_constraint_preconditioner_converges_in_one_step():
    """P_C with P_V = A and P_Q = B A^{-1} B^T - (B A^{-1} B^T - P_Q) reproduces 𝒜
    up to the constant-pressure correction, so P_C^{-1} 𝒜 = I on the range."""
    S, A, Av, Bt, Sch, nv = _ideal_blocks(2, 3)
    C = np.ones_like(Sch) / Sch.shape[0]
    P = np.zeros_like(A)
    P[:nv, :nv] = Av
    P[:nv, nv:] = Bt
    P[nv:, :nv] = Bt.T
    P[nv:, nv:] = -C                                            # B A^{-1} B^T - P_Q with P_Q = S + C
    rng = np.random.default_rng(8)
    b = A @ rng.standard_normal(A.shape[0])
    b[nv:] -= b[nv:].mean()
    x, info = gmres.gmres(lambda v: A @ v, b, lambda v: np.linalg.solve(P, v), tol=1e-10, maxit=10)
    assert info["status"] == "converged" and info["iters"] == 1


@pytest.mark.parametrize("dim,disc,n_el", [(2, "TH", 3), (3, "TH", 2), (2, "RT", 3)])
def test_block_preconditioner_applies_match_dense_inverses(dim, disc, n_el):
    S = stokes.build_uniform(n_el, 2, dim, disc)
    rng = np.random.default_rng(9)
    r = rng.standard_normal(S.n_total)
    PT, PC = stokes.pt_matrix(S), stokes.pc_matrix(S)
    for method in ("fd", "dense"):
        np.testing.assert_allclose(stokes.apply_PT_inv(S, r, method), np.linalg.solve(PT, r), rtol=1e-10,
                                   atol=1e-10 * np.abs(np.linalg.solve(PT, r)).max())
        np.testing.assert_allclose(stokes.apply_PC_inv(S, r, method), np.linalg.solve(PC, r), rtol=1e-10,
                                   atol=1e-10 * np.abs(np.linalg.solve(PC, r)).max())


def test_pt_gmres_on_the_stokes_system():
    """P_T-GMRES and P_C-GMRES reach the tolerance on a small TH system with a
    mean-free pressure right-hand side, in fewer iterations than P_D-MINRES
    (the ordering the paper reports for its mapped domains)."""
    S = stokes.build_uniform(4, 2, 2)
    rng = np.random.default_rng(10)
    b = rng.standard_normal(S.n_total)
    nq = S.block_sizes[-1]
    b[-nq:] -= b[-nq:].mean()
    A = lambda v: stokes.matvec(S, v)
    _, im = minres.minres(A, b, lambda v: stokes.apply_PD_inv(S, v), tol=1e-8, maxit=300, true_check=True)
    for apply in (stokes.apply_PT_inv, stokes.apply_PC_inv):
        x, ig = gmres.gmres(A, b, lambda v: apply(S, v), tol=1e-8, maxit=300, true_check=True)
        assert ig["status"] == "converged" and ig["true_rel"] <= 1e-8
        assert ig["iters"] < im["iters"]


def test_flexible_gmres_solves_and_tracks_the_true_residual():
    rng = np.random.default_rng(11)
    n = 20
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    Mi = np.diag(1.0 / rng.uniform(1.0, 3.0, n))
    b = rng.standard_normal(n)
    x, info = gmres.gmres(lambda v: A @ v, b, lambda v: Mi @ v, tol=1e-12, maxit=n, flexible=True)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)
    hist = []
    for k in range(1, 7):
        hist.clear()
        x, _ = gmres.gmres(lambda v: A @ v, b, lambda v: Mi @ v, tol=0.0, maxit=k, history=hist, flexible=True)
        direct = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert abs(hist[-1] - direct) <= 1e-12 * max(1.0, direct)


def test_flexible_gmres_with_a_varying_preconditioner():
    """The flexible form keeps A Z_j = V_{j+1} H_j for a preconditioner that changes
    from step to step (here: a diagonal perturbed by 1e-3 at every call), so it
    still reaches 1e-10 with an accurate estimate."""
    rng = np.random.default_rng(12)
    n = 40
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    d = rng.uniform(1.0, 3.0, n)
    calls = [0]

    def Pinv(v):
        calls[0] += 1
        return v / (d * (1 + 1e-3 * np.sin(calls[0] + np.arange(n))))
    b = rng.standard_normal(n)
    x, info = gmres.gmres(lambda v: A @ v, b, Pinv, tol=1e-10, maxit=n, flexible=True)
    assert info["status"] == "converged"
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10 * 1.01
