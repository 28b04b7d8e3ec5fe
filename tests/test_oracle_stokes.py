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


def _rt_constants(S):
    """C_pen = 5(alpha + 1) (Sec. 7) with alpha the pressure regularity, h the
    element size: read off the pressure knots, not the velocity spaces."""
    t = S.pres[0].knots
    z = np.unique(t)
    alpha = S.p - int(np.sum(t == z[1]))
    return 5.0 * (alpha + 1), float(np.max(np.diff(z)))


def _rt_compare(S):
    cpen, h = _rt_constants(S)
    A_bf, B_bf = stokes.brute_force_RT(S, cpen, h)
    A = stokes.assembled(S)
    nv = sum(S.block_sizes[:S.dim])
    return (np.abs(A[:nv, :nv] - A_bf).max() / np.abs(A_bf).max(),
            np.abs(A[nv:, :nv] - B_bf).max() / np.abs(B_bf).max(),
            np.abs(A[:nv, nv:] - B_bf.T).max() / np.abs(B_bf).max())


@pytest.mark.parametrize("dim,p,n_el", [(2, 2, 3), (2, 3, 3), (3, 2, 2), (3, 3, 2), (2, 2, (3, 4))])
def test_rt_blocks_vs_brute_force_nitsche_quadrature(dim, p, n_el):
    """Every block of the RT system (A_rs for all r, s, with the Nitsche form
    sigma of eq. theta, and B) equals an element-by-element quadrature of
    a + sigma and b written from their definitions (Sec. 3, eq. RT_dis)."""
    S = stokes.build_uniform(n_el, p, dim, "RT")
    if not np.isscalar(n_el):
        # uneven meshes: the oracle's per-direction h is that direction's span; sigma's h
        # is one number, so compare on the common largest span
        h = max(1.0 / n for n in n_el)
        for k in range(dim):
            for d in range(dim):
                if S.vel[k][d].nitsche:
                    S.vel[k][d].h = h
        cpen, _ = _rt_constants(S)
        A_bf, B_bf = stokes.brute_force_RT(S, cpen, h)
        A = stokes.assembled(S)
        nv = sum(S.block_sizes[:dim])
        assert np.abs(A[:nv, :nv] - A_bf).max() <= 1e-12 * np.abs(A_bf).max()
        assert np.abs(A[nv:, :nv] - B_bf).max() <= 1e-12 * np.abs(B_bf).max()
        return
    ea, eb, ebt = _rt_compare(S)
    assert ea <= 1e-12 and eb <= 1e-12 and ebt <= 1e-12, (ea, eb, ebt)


def _boundary_outer(sa, sb, at, db=0):
    from oracle import splines
    Ba, _ = splines.basis(sa.knots, sa.degree, np.array([at]))
    Bb, Db = splines.basis(sb.knots, sb.degree, np.array([at]))
    return np.outer(Ba[0, sa.keep], (Bb, Db)[db][0, sb.keep])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("mistake", ["drop_nitsche", "penalty_doubled", "consistency_sign",
                                     "nitsche_in_cross_block"])
def test_rt_brute_force_catches_planted_mistakes(monkeypatch, dim, mistake):
    """A mistake planted in the oracle's RT assembly (the Nitsche terms
    dropped, a wrong penalty, a flipped consistency sign, a boundary term put
    into a cross block A_rs) moves it away from the brute-force quadrature by
    far more than the 1e-12 bar."""
    from oracle import univariate as uv
    S = stokes.build_uniform(2, 2, dim, "RT")
    if mistake == "drop_nitsche":
        for k in range(dim):
            for d in range(dim):
                S.vel[k][d].nitsche = False
    elif mistake == "penalty_doubled":
        for k in range(dim):
            for d in range(dim):
                S.vel[k][d].cpen *= 2.0
    elif mistake == "consistency_sign":
        orig = uv.stiffness

        def flipped(s, weight=None, npts=None, tau0=1.0, tau1=1.0):
            if not s.nitsche:
                return orig(s, weight, npts, tau0, tau1)
            # K~ with the consistency terms' sign flipped: K~' = 2 K - K~ + penalty twice
            K0 = uv.mixed(s, 1, s, 1, weight, npts)
            Kn = orig(s, weight, npts, tau0, tau1)
            pen = 2.0 * s.cpen / s.h * (_boundary_outer(s, s, 1.0) + _boundary_outer(s, s, 0.0))
            return 2.0 * K0 - Kn + 2.0 * pen
        monkeypatch.setattr(uv, "stiffness", flipped)
    elif mistake == "nitsche_in_cross_block":
        orig_terms = stokes.a_block_terms

        def moved(S_, r, s):
            terms = orig_terms(S_, r, s)
            if r == s:
                return terms
            # a consistency-type face term of direction s (value of component r's
            # tangential factor times the normal derivative of component s's factor)
            f = [uv.mixed(S_.vel[r][e], 0, S_.vel[s][e], 0) for e in range(S_.dim)]
            f[s] = (_boundary_outer(S_.vel[r][s], S_.vel[s][s], 1.0, db=1)
                    - _boundary_outer(S_.vel[r][s], S_.vel[s][s], 0.0, db=1))
            return terms + [(S_.nu, f)]
        monkeypatch.setattr(stokes, "a_block_terms", moved)
    ea, _, _ = _rt_compare(S)
    assert ea > 1e-3, (mistake, ea)


def test_rt_nitsche_adds_nothing_to_cross_blocks_on_the_cube():
    """The reading that sigma contributes only to A_kk on the cube: the face
    integrals of sigma over the cross pairs (e_r B_i, e_s B_j), r != s, taken
    alone from the brute force (a + sigma minus a), vanish."""
    S = stokes.build_uniform(2, 2, 3, "RT")
    cpen, h = _rt_constants(S)
    A_full, _ = stokes.brute_force_RT(S, cpen, h)
    A_vol, _ = stokes.brute_force_RT(S, 0.0, h, nu=1.0, faces=False)
    sig = A_full - A_vol
    off = np.concatenate([[0], np.cumsum(S.block_sizes[:3])])
    for r in range(3):
        for s in range(3):
            blk = sig[off[r]:off[r + 1], off[s]:off[s + 1]]
            if r == s:
                assert np.abs(blk).max() > 0.1 * np.abs(sig).max()
            else:
                assert np.abs(blk).max() <= 1e-13 * np.abs(sig).max()
