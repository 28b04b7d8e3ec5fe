"""Pins for the Raviart-Thomas parts of oracle.geometry: the RT system on the
identity map with a variable viscosity (Sec. 3 forms, eq. theta with nu at the
face points) and its coefficient-aware preconditioner (Sec. 6, eq. Q_RT, the
Appendix's weighted K~, M~ with the tau(0), tau(1) boundary terms)."""
import numpy as np
import pytest

from oracle import geometry as geo, kron, minres, stokes, univariate as uv
import synth


def _rt(n_el, p):
    return stokes.build_uniform(n_el, p, 3, disc="RT")


def _dense(S, G):
    """Dense [[A, B^T], [B, 0]] by brute-force quadrature of the forms."""
    cpen, h = geo._nitsche_constants(S)
    A, B = stokes.brute_force_RT(S, cpen, h, nu=lambda X: G.nu_of(X))
    nv = A.shape[0]
    full = np.zeros((S.n_total, S.n_total))
    full[:nv, :nv] = A
    full[nv:, :nv] = B
    full[:nv, nv:] = B.T
    return full, A


@pytest.mark.parametrize("contrast", [None, 100.0], ids=["sin_cos_field", "contrast100"])
def test_rt_operator_with_variable_viscosity_vs_brute_force(contrast):
    """Sum-factorized volume forms plus the face-by-face Nitsche form against
    the dense brute-force quadrature of a + sigma and b (all blocks, r != s
    included), and the diagonal used by D_V against the dense diagonal."""
    S = _rt((2, 2, 3), 2)
    G = geo.Grid(S, amp=0.0, contrast=contrast)
    full, A = _dense(S, G)
    rng = np.random.default_rng(31)
    for _ in range(3):
        x = rng.standard_normal(S.n_total)
        np.testing.assert_allclose(geo.operator(S, G, x), full @ x, rtol=0, atol=1e-12 * np.abs(full).max())
    off = np.concatenate([[0], np.cumsum(S.block_sizes[:3])])
    for k in range(3):
        d = geo.diag_A(S, G, k) + geo.nitsche_diag(S, G, k)
        np.testing.assert_allclose(d, np.diag(A)[off[k]:off[k + 1]], rtol=1e-12)


def test_rt_faces_use_the_face_viscosity():
    """Planted in the oracle: the face integrals with nu = 1 instead of nu at the
    face points must disagree with the brute force (the pin above sees nu there)."""
    S = _rt((2, 2, 2), 1)
    G = geo.Grid(S, amp=0.0)
    full, _ = _dense(S, G)
    x = np.random.default_rng(32).standard_normal(S.n_total)
    real_at = G.at

    def at_nu1(E):
        P = real_at(E)
        P.nu = np.ones_like(P.nu)
        return P
    G.at = at_nu1
    y = geo.operator(S, G, x)
    G.at = real_at
    assert np.abs(y - full @ x).max() > 1e-6 * np.abs(full @ x).max()


def test_rt_cube_limit_weighted_pencils_equal_plain():
    """nu = 1 on the identity map: C_k^RT = I + e_k e_k^T, the fit is exact, the
    weighted K~, M~ are the plain ones (the factor 2 of eq. prec3D_RT inside tau),
    D_V = D_Q = 1, and P_D^G = P_D."""
    S = _rt((3, 2, 2), 2)
    G = geo.Grid(S, amp=0.0, nu_const=1.0)
    pdg = geo.PDG(S, G)
    for k in range(3):
        Ks, Ms, _ = pdg.pencils[k]
        K0, M0, coef = stokes.pv_pencils(S, k)
        for d in range(3):
            np.testing.assert_allclose(Ks[d], coef[d] * K0[d], rtol=1e-12, atol=1e-12 * np.abs(K0[d]).max())
            np.testing.assert_allclose(Ms[d], M0[d], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(pdg.DV[k], 1.0, rtol=1e-12)
    np.testing.assert_allclose(pdg.DQ, 1.0, rtol=1e-12)
    r = np.random.default_rng(33).standard_normal(S.n_total)
    np.testing.assert_allclose(pdg.apply(r), stokes.apply_PD_inv(S, r), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("k", [100.0, 1.0e4])
def test_rt_contrast_family_weighted_pencils_equal_the_diagonal_blocks(k):
    """nu_k depends on eta_1 alone on the identity map, so the separable fit of
    diag(C_k^RT) is exact and the Kronecker sum of the Appendix's weighted
    pencils (tau at the quadrature points, tau(0), tau(1) in the K~ boundary
    terms) reproduces A_kk = a + sigma of the brute force; D_V = 1."""
    S = _rt((3, 2, 2), 2)
    G = geo.Grid(S, amp=0.0, contrast=k)
    pdg = geo.PDG(S, G)
    _, A = _dense(S, G)
    off = np.concatenate([[0], np.cumsum(S.block_sizes[:3])])
    for c in range(3):
        Ks, Ms, coef = pdg.pencils[c]
        Akk = A[off[c]:off[c + 1], off[c]:off[c + 1]]
        np.testing.assert_allclose(kron.kron_sum_matrix(Ks, Ms, coef), Akk, rtol=0, atol=1e-11 * np.abs(Akk).max())
        np.testing.assert_allclose(pdg.DV[c], 1.0, rtol=1e-9)


def test_rt_boundary_weights_are_needed(monkeypatch):
    """Planted in the oracle: the K~ boundary terms with tau(0) = tau(1) = 1 (the
    plain pencils' bracket) no longer reproduce A_kk on the contrast family."""
    S = _rt((3, 2, 2), 2)
    G = geo.Grid(S, amp=0.0, contrast=100.0)
    _, A = _dense(S, G)
    real = uv.nitsche_boundary
    monkeypatch.setattr(uv, "nitsche_boundary", lambda s, tau0=1.0, tau1=1.0: real(s))
    pdg = geo.PDG(S, G)
    n0 = S.block_sizes[0]
    Ks, Ms, coef = pdg.pencils[0]
    assert np.abs(kron.kron_sum_matrix(Ks, Ms, coef) - A[:n0, :n0]).max() > 1e-3 * np.abs(A[:n0, :n0]).max()


def test_rt_non_separable_viscosity_diagonals():
    """On the non-separable field nu = 1 + sin(2 pi x1) cos(2 pi x2) / 2 the fit is
    approximate; D_V still makes diag(P_V^G) = diag(A) (faces included) and
    diag(P_Q^G) = diag(Q) (Sec. 6)."""
    S = _rt((2, 3, 2), 2)
    G = geo.Grid(S, amp=0.0)
    pdg = geo.PDG(S, G)
    _, A = _dense(S, G)
    off = np.concatenate([[0], np.cumsum(S.block_sizes[:3])])
    for k in range(3):
        Ks, Ms, _ = pdg.pencils[k]
        P = kron.kron_sum_matrix(Ks, Ms, [1.0, 1.0, 1.0])
        PG = np.sqrt(pdg.DV[k])[:, None] * P * np.sqrt(pdg.DV[k])[None, :]
        np.testing.assert_allclose(np.diag(PG), np.diag(A)[off[k]:off[k + 1]], rtol=1e-12)
        # the fit is not exact here: the weighted pencils differ from A_kk
        Akk = A[off[k]:off[k + 1], off[k]:off[k + 1]]
        assert np.abs(P - Akk).max() > 1e-4 * np.abs(Akk).max()


def test_c_matrix_rt_is_the_piola_symmetric_gradient_form():
    """For a constant Jacobian the RT basis e_k B pushed forward by Piola,
    v = J e_k B / det J, has grad_x v = (J e_k / det J)(J^{-T} grad_eta B)^T, and
    int 2 nu grad^s v_i : grad^s v_j dx = g_i^T C_k^RT g_j |...| deta pointwise
    (eq. Q_RT without its Hessian terms, which vanish for an affine map)."""
    rng = np.random.default_rng(34)
    for trial in range(20):
        J = np.eye(3) + 0.4 * rng.standard_normal((3, 3))
        det = np.linalg.det(J)
        if abs(det) < 0.2:
            continue
        Jinv = np.linalg.inv(J)
        nu = 0.5 + rng.random()
        k = trial % 3
        C = geo.c_matrix_rt(J, np.array(det), Jinv, np.array(nu), k)
        for _ in range(4):
            gi, gj = rng.standard_normal(3), rng.standard_normal(3)
            Gi = np.outer(J[:, k] / det, Jinv.T @ gi)
            Gj = np.outer(J[:, k] / det, Jinv.T @ gj)
            Si, Sj = 0.5 * (Gi + Gi.T), 0.5 * (Gj + Gj.T)
            brute = 2.0 * nu * np.sum(Si * Sj) * abs(det)
            assert abs(gi @ C @ gj - brute) <= 1e-12 * max(1.0, abs(brute))
    # identity map: C_k^RT = nu (I + e_k e_k^T)
    for k in range(3):
        C = geo.c_matrix_rt(np.eye(3), np.array(1.0), np.eye(3), np.array(2.5), k)
        np.testing.assert_allclose(C, 2.5 * (np.eye(3) + np.outer(np.eye(3)[k], np.eye(3)[k])), atol=1e-15)


def test_fit_at_reproduces_a_separable_field_on_the_faces():
    """The fit's update evaluated on a face returns the direction-d factor there:
    on an exactly separable field exp(f_end + f_a + f_b) equals the field on the face."""
    rng = np.random.default_rng(35)
    n = (6, 5, 7)
    g = [lambda t, a=a: np.sin(3 * t + a) + a * t for a in (0.3, 1.1, -0.7)]
    pts = [np.sort(rng.random(m)) for m in n]
    c = np.exp(g[0](pts[0])[:, None, None] + g[1](pts[1])[None, :, None] + g[2](pts[2])[None, None, :])
    f = geo.separable_fit(c)
    for d in range(3):
        for t in (0.0, 1.0):
            axes = [np.array([t]) if e == d else pts[e] for e in range(3)]
            cf = np.exp(g[0](axes[0])[:, None, None] + g[1](axes[1])[None, :, None] + g[2](axes[2])[None, None, :])
            fd = geo.fit_at(np.log(cf), f, d)
            shp = [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]
            rec = np.exp(fd + sum(f[e].reshape(shp[e]) for e in range(3) if e != d))
            np.testing.assert_allclose(rec, cf, rtol=1e-12)


def test_rt_geometry_aware_preconditioner_on_the_contrast_family():
    """P_D ignores nu; P_D^G carries it in the weighted pencils and the diagonal
    scalings. On the RT contrast family P_D^G-MINRES needs far fewer iterations
    than P_D-MINRES, and both reach the tolerance (the true residual; MINRES
    continues past the recurrence estimate until it does)."""
    S = _rt(3, 1)
    G = geo.Grid(S, amp=0.0, contrast=100.0)
    pdg = geo.PDG(S, G)
    A = lambda v: geo.operator(S, G, v)
    b = synth.rhs(7, S.block_sizes)
    its = {}
    for name, apply in (("PDG", pdg.apply), ("PD", lambda v: stokes.apply_PD_inv(S, v))):
        x, info = minres.minres(A, b, apply, tol=1e-8, maxit=3000, true_check=True)
        assert np.linalg.norm(b - A(x)) <= 1e-8 * np.linalg.norm(b)
        its[name] = info["iters"]
    assert its["PDG"] <= 0.5 * its["PD"], its
