"""Pins for oracle.geometry (paper Sec. 3 mapped forms, Sec. 6, Appendix)."""
import numpy as np
import pytest

from oracle import geometry as geo, kron, stokes
import synth


def _S(n_el, p):
    return stokes.build([synth.open_uniform_knots(n, p) for n in (n_el if not np.isscalar(n_el) else (n_el,) * 3)], p)


def test_det_closed_form_and_jacobian():
    rng = np.random.default_rng(0)
    eta = rng.random((50, 3))
    x, J, det, Jinv = geo.geometry(eta)
    np.testing.assert_allclose(det, np.linalg.det(J), rtol=1e-14)
    # J by central differences of the map
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        xp, *_ = geo.geometry(eta + e)
        xm, *_ = geo.geometry(eta - e)
        np.testing.assert_allclose(J[:, :, j], (xp - xm) / (2 * h), atol=1e-8)
    # det J range of the 0.1 sine bump: 1 +- 0.1 pi sqrt(4/3) (max of the gradient sum)
    g = np.stack(np.meshgrid(*[np.linspace(0, 1, 41)] * 3, indexing="ij"), -1)
    _, _, d, _ = geo.geometry(g)
    assert 0.6 < d.min() < 0.7 and 1.3 < d.max() < 1.4


def test_sum_factorized_matvec_vs_brute_force():
    S = _S(2, 1)
    G = geo.Grid(S)
    A, B = geo.brute_force(S, G)
    nv = 3 * S.block_sizes[0]
    full = np.zeros((S.n_total, S.n_total))
    full[:nv, :nv] = A
    full[nv:, :nv] = B
    full[:nv, nv:] = B.T
    rng = np.random.default_rng(3)
    for _ in range(3):
        x = rng.standard_normal(S.n_total)
        np.testing.assert_allclose(geo.matvec(S, G, x), full @ x, atol=1e-12 * np.abs(full).max() * 10)
    np.testing.assert_allclose(A, A.T, atol=1e-13 * np.abs(A).max())


def test_identity_limit_is_the_cube_operator():
    S = _S(3, 2)
    G = geo.Grid(S, amp=0.0, nu_const=1.0)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(S.n_total)
    np.testing.assert_allclose(geo.matvec(S, G, x), stokes.matvec(S, x), atol=1e-11)


def test_separable_fit_exact_on_separable_field():
    rng = np.random.default_rng(1)
    g = [rng.standard_normal(n) for n in (7, 5, 6)]
    c = np.exp(g[0][:, None, None] + g[1][None, :, None] + g[2][None, None, :])
    f = geo.separable_fit(c)
    rec = np.exp(f[0][:, None, None] + f[1][None, :, None] + f[2][None, None, :])
    np.testing.assert_allclose(rec, c, rtol=1e-12)


def test_separable_fit_reaches_the_closed_form_distance_on_a_bilinear_field():
    """On a tensor grid, log c = a x y + (separable terms) is at sup-norm distance
    exactly a (x_max - x_min)(y_max - y_min) / 4 from the sums f1 + f2 + f3: every
    sum cancels in the alternating sum over the four corners (x_min|x_max, y_min|y_max)
    while a x y leaves a dx dy there (the lower bound), and a (x - c_x)(y - c_y) with
    c the grid midpoints attains it. The midrange sweeps must reach that optimum; a
    mean in place of the midrange misses it on the uneven grid used here."""
    rng = np.random.default_rng(3)
    x, y, z = np.sort(rng.uniform(-1, 2, 7)), np.sort(rng.uniform(0.5, 3, 5)), rng.uniform(0, 1, 4)
    a = 0.7
    g = [rng.standard_normal(n) for n in (7, 5, 4)]
    dist = a * np.ptp(x) * np.ptp(y) / 4
    bilinear = a * x[:, None, None] * y[None, :, None]
    cx, cy = 0.5 * (x.max() + x.min()), 0.5 * (y.max() + y.min())
    optimal = a * (x[:, None, None] - cx) * (y[None, :, None] - cy) * np.ones((1, 1, 4))
    for L, exact_residual in ((bilinear + g[0][:, None, None] + g[2][None, None, :], True),
                              (bilinear + g[0][:, None, None] + g[1][None, :, None] + g[2][None, None, :], False)):
        f = geo.separable_fit(np.exp(L))
        R = L - f[0][:, None, None] - f[1][None, :, None] - f[2][None, None, :]
        assert abs(np.abs(R).max() - dist) <= 1e-12 * dist
        if exact_residual:   # separable terms only in x and z: the optimal residual itself
            np.testing.assert_allclose(R, optimal, atol=1e-12)
    # the same bound in the (x, z) pair
    L = a * x[:, None, None] * z[None, None, :] + g[1][None, :, None]
    f = geo.separable_fit(np.exp(L))
    R = L - f[0][:, None, None] - f[1][None, :, None] - f[2][None, None, :]
    assert abs(np.abs(R).max() - a * np.ptp(x) * np.ptp(z) / 4) <= 1e-12
    # a mean in place of the midrange would leave a larger error on this grid
    mean_fit = np.abs(a * (x[:, None] - x.mean()) * (y[None, :] - y.mean())).max()
    assert mean_fit > 1.1 * dist


def test_fit_never_increases_the_sup_error():
    S = _S(3, 2)
    G = geo.Grid(S)
    L = np.log(geo.c_diag(G, 0)[1])
    errs = []
    for sw in (1, 2, 4, 8, 12):
        f = geo.separable_fit(np.exp(L), sweeps=sw)
        errs.append(np.abs(L - f[0][:, None, None] - f[1][None, :, None] - f[2][None, None, :]).max())
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))


def test_cube_limit_weighted_pencils_equal_plain():
    S = _S(3, 2)
    G = geo.Grid(S, amp=0.0, nu_const=1.0)
    pdg = geo.PDG(S, G)
    for k in range(3):
        Ks, Ms, _ = pdg.pencils[k]
        K0, M0, coef = stokes.pv_pencils(S, k)
        for d in range(3):
            np.testing.assert_allclose(Ks[d], coef[d] * K0[d], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(Ms[d], M0[d], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(pdg.DV[k], 1.0, rtol=1e-12)
    np.testing.assert_allclose(pdg.DQ, 1.0, rtol=1e-12)
    r = np.random.default_rng(2).standard_normal(S.n_total)
    np.testing.assert_allclose(pdg.apply(r), stokes.apply_PD_inv(S, r), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind", ["sine_bump", "annulus"])
def test_scaled_diagonals_match_operator_diagonals(kind):
    """diag(P_V^G) = diag(A) and diag(P_Q^G) = diag(Q) by construction (Sec. 6)."""
    S = _S(2, 1)
    G = geo.Grid(S, geometry_kind=kind)
    pdg = geo.PDG(S, G)
    A, _ = geo.brute_force(S, G)
    nv = S.block_sizes[0]
    for k in range(3):
        Ks, Ms, _ = pdg.pencils[k]
        Pk = kron.kron_sum_matrix(Ks, Ms, [1.0, 1.0, 1.0])
        PG = np.sqrt(pdg.DV[k])[:, None] * Pk * np.sqrt(pdg.DV[k])[None, :]
        np.testing.assert_allclose(np.diag(PG), np.diag(A)[k * nv:(k + 1) * nv], rtol=1e-12)


@pytest.mark.parametrize("kind", ["sine_bump", "annulus"])
def test_theorem2_pressure_mass_bounds(kind):
    """lambda(P_Q^{-1} Q) lies in [min |det J|/nu, max |det J|/nu] (Theorem 2, Remark)."""
    S = _S(2, 2)
    G = geo.Grid(S, geometry_kind=kind)
    T = [G.table(S.pres[d], d, False) for d in range(3)]
    F = (G.W * np.abs(G.det) / G.nu).reshape(-1)
    Bq = np.einsum("ap,bq,cr->cbapqr", T[0], T[1], T[2]).reshape(S.block_sizes[3], -1)
    Q = (Bq * F) @ Bq.T
    PQ = kron.kron_matrix(stokes.pq_factors(S))
    lam = np.linalg.eigvals(np.linalg.solve(PQ, Q)).real
    ratio = np.abs(G.det) / G.nu
    assert lam.min() >= ratio.min() * (1 - 1e-10)
    assert lam.max() <= ratio.max() * (1 + 1e-10)
    np.testing.assert_allclose(np.sort(np.diag(Q)), np.sort(geo.diag_Q(S, G)), rtol=1e-12)


def test_operator_row_vs_brute_force():
    S = _S(2, 1)
    G = geo.Grid(S)
    A, B = geo.brute_force(S, G)
    nv = 3 * S.block_sizes[0]
    full = np.zeros((S.n_total, S.n_total))
    full[:nv, :nv] = A
    full[nv:, :nv] = B
    full[:nv, nv:] = B.T
    n = [S.vel[0][d].n for d in range(3)]
    npr = [S.pres[d].n for d in range(3)]
    off = np.concatenate([[0], np.cumsum(S.block_sizes)])
    for blk, m in [(0, (1, 0, 2)), (2, (2, 2, 0)), (1, (0, 1, 1)), (3, (1, 2, 0)), (3, (0, 0, 0))]:
        sp = n if blk < 3 else npr
        row = off[blk] + (m[2] * sp[1] + m[1]) * sp[0] + m[0]
        ent = geo.operator_row(S, G, blk, m)
        dense = np.zeros(S.n_total)
        for c, v in ent.items():
            dense[c] = v
        np.testing.assert_allclose(dense, full[row], atol=1e-13 * np.abs(full).max())



def test_mapped_block_preconditioners_match_dense_inverses():
    """P_T^G and P_C^G (Sec. 6 blocks in eq. P_T, eq. P_C) applied through the
    oracle against the dense matrices assembled from brute-force quadrature of
    the mapped operator and the dense P_V^G, P_Q^G."""
    from oracle import kron, stokes
    S = stokes.build_uniform((2, 2, 3), 1, 3)
    G = geo.Grid(S)
    pdg = geo.PDG(S, G)
    A_bf, B_bf = geo.brute_force(S, G)
    nv = sum(S.block_sizes[:3])
    PV = np.zeros((nv, nv))
    off = np.concatenate([[0], np.cumsum(S.block_sizes[:3])])
    for k in range(3):
        Ks, Ms, coef = pdg.pencils[k]
        sc = np.sqrt(pdg.DV[k])
        PV[off[k]:off[k + 1], off[k]:off[k + 1]] = sc[:, None] * kron.kron_sum_matrix(Ks, Ms, coef) * sc[None, :]
    sq = np.sqrt(pdg.DQ)
    PQ = sq[:, None] * kron.kron_matrix(pdg.Mp) * sq[None, :]
    PT = np.block([[PV, B_bf.T], [np.zeros_like(B_bf), -PQ]])
    PC = np.block([[PV, B_bf.T], [B_bf, B_bf @ np.linalg.solve(PV, B_bf.T) - PQ]])
    rng = np.random.default_rng(14)
    r = rng.standard_normal(S.n_total)
    for apply, P in ((geo.apply_PTG_inv, PT), (geo.apply_PCG_inv, PC)):
        ref = np.linalg.solve(P, r)
        np.testing.assert_allclose(apply(S, G, pdg, r), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("k", [1.0, 100.0, 1.0e4])
def test_viscosity_contrast_family_and_exact_fit_on_the_cube(k):
    """nu_k(x) = 1 + (k - 1)(1 - cos(2 pi x1)) / 2 takes values in [1, k]; on the
    identity map it depends on eta1 alone, so the separable fit is exact and the
    weighted Kronecker sum equals the velocity diagonal block A_kk (D_V = 1)."""
    x = np.stack(np.meshgrid(np.linspace(0, 1, 9), np.linspace(0, 1, 5), [0.3], indexing="ij"), -1)
    nu = geo.viscosity(x, k)
    assert nu.min() >= 1.0 - 1e-15 and nu.max() <= k * (1 + 1e-15)
    S = stokes.build_uniform((3, 2, 2), 2, 3)
    G = geo.Grid(S, amp=0.0, contrast=k)
    pdg = geo.PDG(S, G)
    A_bf, _ = geo.brute_force(S, G)
    off = np.concatenate([[0], np.cumsum(S.block_sizes[:3])])
    for c in range(3):
        Ks, Ms, coef = pdg.pencils[c]
        np.testing.assert_allclose(pdg.DV[c], 1.0, rtol=1e-9)
        Akk = A_bf[off[c]:off[c + 1], off[c]:off[c + 1]]
        np.testing.assert_allclose(kron.kron_sum_matrix(Ks, Ms, coef), Akk, atol=1e-9 * np.abs(Akk).max())


# ---------------------------------------------------------------- eighth of a thick annulus

def test_annulus_map_closed_forms():
    """Polar map of the eighth of a thick annulus (Sec. 7: radii 1 and 2, height 1):
    det J = pi r / 4, J by central differences, boundary faces on the circles and
    planes, quadrature volume 3 pi / 8 and moment int x1 dx = 7 sqrt(2) / 6."""
    rng = np.random.default_rng(7)
    eta = rng.random((60, 3))
    x, J, det, Jinv = geo.geometry(eta, kind="annulus")
    np.testing.assert_allclose(det, np.pi * (1 + eta[:, 0]) / 4, rtol=1e-14)
    np.testing.assert_allclose(det, np.linalg.det(J), rtol=1e-13)
    np.testing.assert_allclose(np.einsum("qab,qbc->qac", J, Jinv), np.broadcast_to(np.eye(3), J.shape), atol=1e-14)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        xp, *_ = geo.geometry(eta + e, kind="annulus")
        xm, *_ = geo.geometry(eta - e, kind="annulus")
        np.testing.assert_allclose(J[:, :, j], (xp - xm) / (2 * h), atol=1e-8)
    t = rng.random(20)
    for face, rad in ((0.0, 1.0), (1.0, 2.0)):
        xf, *_ = geo.geometry(np.stack([np.full(20, face), t, t[::-1]], -1), kind="annulus")
        np.testing.assert_allclose(np.hypot(xf[:, 0], xf[:, 1]), rad, rtol=1e-14)
    x0, *_ = geo.geometry(np.stack([t, np.zeros(20), t], -1), kind="annulus")
    x1, *_ = geo.geometry(np.stack([t, np.ones(20), t], -1), kind="annulus")
    assert np.all(x0[:, 1] == 0.0)
    np.testing.assert_allclose(x1[:, 0], x1[:, 1], rtol=1e-14)
    S = _S(4, 2)
    G = geo.Grid(S, geometry_kind="annulus")
    assert np.all(G.nu == 1.0)
    np.testing.assert_allclose(np.sum(G.W * G.det), 3 * np.pi / 8, rtol=1e-14)
    np.testing.assert_allclose(np.sum(G.W * G.det * G.x[..., 0]), 7 * np.sqrt(2) / 6, rtol=1e-10)


def test_annulus_chain_rule():
    """J^{-T} grad_eta (f o G) = grad_x f for f = x1^2 x2 + x2 x3 - x1 x3^2 (the
    eta-gradient by central differences, independent of J)."""
    f = lambda x: x[..., 0] ** 2 * x[..., 1] + x[..., 1] * x[..., 2] - x[..., 0] * x[..., 2] ** 2
    gf = lambda x: np.stack([2 * x[..., 0] * x[..., 1] - x[..., 2] ** 2, x[..., 0] ** 2 + x[..., 2],
                             x[..., 1] - 2 * x[..., 0] * x[..., 2]], -1)
    eta = np.random.default_rng(8).random((40, 3)) * 0.98 + 0.01
    x, _, _, Jinv = geo.geometry(eta, kind="annulus")
    h = 1e-5
    ge = np.zeros_like(eta)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        ge[:, a] = (f(geo.geometry(eta + e, kind="annulus")[0]) - f(geo.geometry(eta - e, kind="annulus")[0])) / (2 * h)
    np.testing.assert_allclose(np.einsum("qa,qac->qc", ge, Jinv), gf(x), atol=1e-8)


@pytest.mark.parametrize("kind", ["sine_bump", "annulus"])
def test_divergence_of_zero_trace_fields_integrates_to_zero(kind):
    """B^T 1 = 0: int div v dx = 0 for every v vanishing on the boundary (any map).
    With a high-order rule the quadrature error is negligible, so a transposed J^{-1}
    or a missing det J factor shows."""
    S = _S(3, 2)
    G = geo.Grid(S, npts=14, geometry_kind=kind)
    nv = 3 * S.block_sizes[0]
    x = np.zeros(S.n_total)
    x[nv:] = 1.0
    y = geo.matvec(S, G, x)
    x[nv:] = np.random.default_rng(4).standard_normal(S.n_total - nv)
    scale = np.abs(geo.matvec(S, G, x)[:nv]).max()
    assert np.abs(y[:nv]).max() <= 1e-12 * scale


def test_annulus_sum_factorized_matvec_vs_brute_force():
    S = _S(2, 1)
    G = geo.Grid(S, geometry_kind="annulus")
    A, B = geo.brute_force(S, G)
    nv = 3 * S.block_sizes[0]
    full = np.zeros((S.n_total, S.n_total))
    full[:nv, :nv] = A
    full[nv:, :nv] = B
    full[:nv, nv:] = B.T
    rng = np.random.default_rng(9)
    for _ in range(3):
        x = rng.standard_normal(S.n_total)
        np.testing.assert_allclose(geo.matvec(S, G, x), full @ x, atol=1e-12 * np.abs(full).max() * 10)
    np.testing.assert_allclose(A, A.T, atol=1e-13 * np.abs(A).max())
    assert np.all(np.linalg.eigvalsh(A) > 0)


@pytest.mark.parametrize("kind", ["sine_bump", "annulus"])
def test_theorem1_velocity_bounds(kind):
    """Theorem 1 with the Korn constants 1/2 (Sec. 5, TH): the eigenvalues of P_V^{-1} A
    lie in [nu_min inf(|det J| / ||J||^2) / 2, 2 nu_max sup(|det J| ||J^{-1}||^2)]. The
    upper bound holds pointwise at the quadrature points (|grad^s v| <= |grad v|), so
    exactly; the lower one rests on Korn's identity, exact only for exact integration,
    so it is checked with a 10% margin on these non-polynomial maps."""
    import scipy.linalg
    S = _S(2, 1)
    G = geo.Grid(S, geometry_kind=kind)
    A, _ = geo.brute_force(S, G)
    blocks = []
    for k in range(3):
        K0, M0, coef = stokes.pv_pencils(S, k)
        blocks.append(kron.kron_sum_matrix(K0, M0, coef))
    PV = scipy.linalg.block_diag(*blocks)
    lam = scipy.linalg.eigh(A, PV, eigvals_only=True)
    J, Ji = G.J.reshape(-1, 3, 3), G.Jinv.reshape(-1, 3, 3)
    det = np.abs(G.det.reshape(-1))
    lo = 0.5 * G.nu.min() * np.min(det / np.linalg.norm(J, 2, axis=(1, 2)) ** 2)
    hi = 2.0 * G.nu.max() * np.max(det * np.linalg.norm(Ji, 2, axis=(1, 2)) ** 2)
    assert lam.max() <= hi * (1 + 1e-10)
    assert lam.min() >= 0.9 * lo
