"""Pins for oracle.stokes (paper Sec. 3 forms, Sec. 5 P_V / P_Q, Sec. 7 A_kk = P_V,k)."""
import numpy as np
import pytest

from oracle import kron, stokes


@pytest.mark.parametrize("dim,p,n_el,velocity", [(2, 1, 2, "th"), (2, 2, 2, "th"), (3, 1, 2, "th"),
                                                 (2, 2, 3, "max_smooth"), (3, 2, 2, "max_smooth")])
def test_kronecker_blocks_vs_brute_force_quadrature(dim, p, n_el, velocity):
    S = stokes.build_uniform(n_el, p, dim, velocity=velocity)
    A_bf, B_bf = stokes.brute_force_TH(S)
    A = stokes.assembled(S)
    nv = S.block_sizes[0] * dim
    np.testing.assert_allclose(A[:nv, :nv], A_bf, atol=1e-12 * np.abs(A_bf).max())
    np.testing.assert_allclose(A[nv:, :nv], B_bf, atol=1e-12 * np.abs(B_bf).max())
    np.testing.assert_allclose(A[:nv, nv:], B_bf.T, atol=1e-12 * np.abs(B_bf).max())
    assert np.all(A[nv:, nv:] == 0)


@pytest.mark.parametrize("dim,disc,velocity", [(2, "TH", "th"), (3, "TH", "th"), (2, "RT", "th"),
                                               (3, "RT", "th"), (2, "TH", "max_smooth"),
                                               (3, "TH", "max_smooth")])
def test_symmetry_nullspace_and_matvec(dim, disc, velocity):
    S = stokes.build_uniform(3 if dim == 3 else 4, 2, dim, disc, velocity=velocity)
    A = stokes.assembled(S)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    # constant pressure is in the kernel: B^T 1 = 0 (partition of unity + v = 0 on the boundary)
    x = np.zeros(S.n_total)
    x[-S.block_sizes[-1]:] = 1.0
    assert np.abs(A @ x).max() < 1e-12
    rng = np.random.default_rng(2)
    y = rng.standard_normal(S.n_total)
    np.testing.assert_allclose(stokes.matvec(S, y), A @ y, atol=1e-11 * np.abs(A @ y).max())
    # A_kk equals P_{V,k} on the identity map
    off = np.concatenate([[0], np.cumsum(S.block_sizes)])
    for k in range(dim):
        np.testing.assert_allclose(A[off[k]:off[k + 1], off[k]:off[k + 1]], stokes.pv_matrix(S, k), atol=0)


@pytest.mark.parametrize("disc,dim", [("TH", 2), ("RT", 2), ("RT", 3)])
def test_preconditioner_blocks_spd(disc, dim):
    S = stokes.build_uniform(3, 2, dim, disc)
    for k in range(dim):
        assert np.linalg.eigvalsh(stokes.pv_matrix(S, k)).min() > 0
    assert np.linalg.eigvalsh(kron.kron_matrix(stokes.pq_factors(S))).min() > 0


@pytest.mark.parametrize("dim,n_el", [(2, 4), (3, 3)])
def test_rt_divergence_lands_in_pressure_space(dim, n_el):
    """RT (Sec. 2.2.2): d/d eta_k of the direction-k factor space is the pressure
    space, so the velocity-pressure coupling is B = -P_Q D with D the exact
    discrete divergence; hence P_Q^{-1} B has integer-free entries that
    reproduce the divergence of a field exactly."""
    S = stokes.build_uniform(n_el, 2, dim, "RT")
    A = stokes.assembled(S)
    nv = sum(S.block_sizes[:dim])
    B = A[nv:, :nv]
    D = -np.linalg.solve(kron.kron_matrix(stokes.pq_factors(S)), B)
    # a velocity field with zero discrete divergence has B v = 0 and D v = 0 simultaneously
    ns = np.linalg.svd(B)[2][np.linalg.matrix_rank(B):]
    assert np.abs(D @ ns.T).max() < 1e-9
    # rank of B: all pressures except the constant
    assert np.linalg.matrix_rank(B) == S.block_sizes[-1] - 1


@pytest.mark.parametrize("n_el,p", [(4, 2), (5, 3), (64, 3)])
def test_max_smooth_velocity_dimensions(n_el, p):
    """Degree p+1 with simple interior breakpoints: n_el + p + 1 functions per
    direction, n_el + p - 1 after Dirichlet removal (66 at 64 elements, p = 3);
    the paper's TH space keeps 2 n_el + p - 2 (129)."""
    S = stokes.build_uniform(n_el, p, 2, velocity="max_smooth")
    assert S.vel[0][0].n == n_el + p - 1
    assert S.pres[0].n == n_el + p
    T = stokes.build_uniform(n_el, p, 2)
    assert T.vel[0][0].n == 2 * n_el + p - 2


@pytest.mark.parametrize("dim,n_el,expected", [(2, 4, 2), (2, 8, 2), (3, 2, 11), (3, 3, 14)])
def test_max_smooth_velocity_is_not_inf_sup_stable(dim, n_el, expected):
    """Reading of the 64^3 size (paper Sec. 7 versus the TH construction of
    Sec. 2.2.1): the maximal-smoothness velocity space on the pressure mesh
    leaves pressures outside the range of B beyond the constant (2D: one, 3D:
    3 n_el + 5), so its Stokes matrix is singular on them and the pair cannot
    stand in for the paper's; the paper's space (every breakpoint repeated)
    leaves only the constant."""
    for velocity, want in (("max_smooth", expected), ("th", 1)):
        S = stokes.build_uniform(n_el, 2, dim, velocity=velocity)
        A = stokes.assembled(S)
        nv = sum(S.block_sizes[:dim])
        B = A[nv:, :nv]
        rank = np.linalg.matrix_rank(B, tol=1e-10 * np.abs(B).max())
        assert B.shape[0] - rank == want
