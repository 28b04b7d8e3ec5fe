"""Mapped geometry, variable viscosity and the geometry-aware preconditioner
P_D^G (paper Sec. 3 eq. Akk_TH / Q_TH, Sec. 6, Appendix). Oracle: test
infrastructure only.

Maps (analytic stand-ins for the paper's spline maps, reading A18):
  sine bump   G(eta) = eta + a sin(pi eta1) sin(pi eta2) sin(pi eta3) (1, 1, 1),
              a = 0.1, so J = I + 1 (a grad s)^T and det J = 1 + a (1 . grad s);
              viscosity nu(x) = 1 + 0.5 sin(2 pi x1) cos(2 pi x2) at x = G(eta).
  annulus     the eighth of a thick annulus of Sec. 7 (inner radius 1, outer
              radius 2, height 1, opening angle pi/4) in polar form:
              r = 1 + eta1, theta = pi eta2 / 4, x = (r cos theta, r sin theta,
              eta3), so det J = pi r / 4; viscosity nu = 1 (constant, as in the
              paper's test). Its P_D lacks the geometry while P_D^G has it.

Operator on the mapped domain (TH push-forward phi = e_r B o G^{-1}):
    a(w, v) = int 2 nu grad^s w : grad^s v,   b(v, q) = -int q div v
with grad_x B = J^{-T} grad_eta B. Quadrature: Gauss with p+2 points per
element and direction.

P_D^G (Sec. 6): P_V^G = D_V^{1/2} P~_V D_V^{1/2} with P~_{V,k} the Kronecker
sum of the weighted pencils (K^k_d with tau^k_d, M^k_d with mu^k_d,
Appendix), [D_V]_ii = A_ii / (P~_V)_ii; P_Q^G = D_Q^{1/2} P_Q D_Q^{1/2},
[D_Q]_ii = Q_ii / (P_Q)_ii with Q the nu^{-1} |det J| weighted pressure mass.

Separable approximation (reading A9; the paper cites Diliberto-Straus /
Wachspress without spelling out the steps): each diagonal entry c^k_jj > 0
of C_k = nu (J^{-1} J^{-T} + D_k D_k^T) |det J| is fitted at the quadrature
points as exp(f1(eta1) + f2(eta2) + f3(eta3)) by the Diliberto-Straus
alternating midrange iteration on log c^k_jj (a fixed 12 sweeps, each
direction in turn: f_d = (max + min)/2 of the residual over the other two
variables). Each fit is normalized so that its two non-own factors have
zero mean log over the quadrature points; then tau^k_j = exp(f^{k,j}_j) and
mu^k_d = exp(mean of f^{k,j}_d over the two j != d). The D_V scaling absorbs
what the fit misses.

Raviart-Thomas on the identity map with a variable viscosity (the RT push-
forward by Piola on a non-trivial map is not built): the volume forms above
with the component-wise RT spaces, plus the Nitsche form sigma of eq. theta
face by face with nu at the face points (penalty C_pen/h_d on the faces normal
to e_d). P_D^G for RT: the diagonal entries of C_k^RT = nu |det J| J^{-1}
(||R_k||^2 I + R_k R_k^T) J^{-T}, R_k = J e_k / det J (eq. Q_RT), fitted as
above; the weighted K~ of the tangential directions carry the Nitsche bracket
with tau^k_d(0), tau^k_d(1) (Appendix). Reading: the fit lives on the
quadrature points as the Appendix says; tau at eta_d = 0, 1 is the fit's own
direction-d update evaluated on those faces (fit_at), which leaves the
interior fit unchanged and is exact for separable fields. D_V adds sigma's
diagonal to diag(A); Q^RT weighs the pressure mass with |det J|^{-1} / nu.

Pins (tests/test_oracle_geometry.py): brute-force element quadrature of the
symmetric-gradient form and of b vs. the sum-factorized matvec (both maps);
amplitude 0 with nu = 1 reproduces the cube operator; det J closed form vs.
numpy.linalg.det; on the annulus the quadrature volume 3 pi / 8 and the
moment int x1 dx = 7 sqrt(2) / 6 in closed form, and the chain rule
J^{-T} grad_eta (f o G) = grad_x f for polynomials f; the fit reproduces an exactly separable field,
and on the non-separable field a x y (plus separable terms) on an uneven tensor grid
it reaches the closed-form sup-norm distance a (x_max - x_min)(y_max - y_min) / 4; on the cube
P~_V = P_V and D_V = I; diag(P_V^G) = diag(A), diag(P_Q^G) = diag(Q);
Theorem 2 spectral bounds of P_Q^{-1} Q and Theorem 1 bounds of P_V^{-1} A
(Korn constants 1/2), on both maps. The fit on the mapped domains' own
fields has no closed form: there it is pinned only through the separable
and bilinear cases above (the CUDA path runs the same algorithm).
RT pins (tests/test_oracle_rt_geometry.py): the RT operator with variable nu
(volume + faces) and its diagonal vs. the dense brute-force quadrature of a +
sigma and b (a non-separable and a separable field; a planted nu = 1 on the
faces fails it); on the contrast family (nu depends on eta_1 alone) the
Kronecker sum of the weighted RT pencils equals the brute-force A_kk and D_V
= 1 (a planted tau(0) = tau(1) = 1 fails it); nu = 1 reduces P_D^G to P_D;
C_k^RT vs. the Piola symmetric-gradient form for constant Jacobians and its
identity-map closed form; fit_at reproduces separable fields on the faces;
P_D^G-MINRES beats P_D-MINRES on the contrast family.
"""
import numpy as np

from . import kron, splines, stokes, univariate as uv

AMP = 0.1
SWEEPS = 12


# ---------------------------------------------------------------- map and viscosity

def bump(eta, amp=AMP):
    """s(eta) = amp sin(pi e1) sin(pi e2) sin(pi e3) and its gradient (..., 3)."""
    e1, e2, e3 = eta[..., 0], eta[..., 1], eta[..., 2]
    s1, s2, s3 = np.sin(np.pi * e1), np.sin(np.pi * e2), np.sin(np.pi * e3)
    c1, c2, c3 = np.cos(np.pi * e1), np.cos(np.pi * e2), np.cos(np.pi * e3)
    s = amp * s1 * s2 * s3
    g = amp * np.pi * np.stack([c1 * s2 * s3, s1 * c2 * s3, s1 * s2 * c3], axis=-1)
    return s, g


def annulus(eta):
    """The eighth of a thick annulus: x, J, det J, J^{-1} of the polar map."""
    r = 1.0 + eta[..., 0]
    th = 0.25 * np.pi * eta[..., 1]
    c, s = np.cos(th), np.sin(th)
    x = np.stack([r * c, r * s, eta[..., 2]], axis=-1)
    J = np.zeros(eta.shape[:-1] + (3, 3))
    J[..., 0, 0], J[..., 1, 0] = c, s                                   # d x / d eta1 (radial)
    J[..., 0, 1], J[..., 1, 1] = -0.25 * np.pi * r * s, 0.25 * np.pi * r * c   # d x / d eta2 (angular)
    J[..., 2, 2] = 1.0
    det = 0.25 * np.pi * r
    return x, J, det, np.linalg.inv(J)


def geometry(eta, amp=AMP, kind="sine_bump"):
    """x = G(eta), J (..., 3, 3) with J_ij = d x_i / d eta_j, det J, J^{-1}."""
    if kind == "annulus":
        return annulus(eta)
    if kind != "sine_bump":
        raise ValueError("unknown geometry %r" % (kind,))
    s, g = bump(eta, amp)
    x = eta + s[..., None]
    J = np.eye(3) + np.ones(3)[:, None] * g[..., None, :]
    det = 1.0 + g.sum(axis=-1)
    Jinv = np.linalg.inv(J)
    return x, J, det, Jinv


def viscosity(x, contrast=None):
    """nu(x) = 1 + 0.5 sin(2 pi x1) cos(2 pi x2); with a contrast k >= 1 the
    one-coordinate family nu(x) = 1 + (k - 1)(1 - cos(2 pi x1)) / 2, values in
    [1, k] (the analytic stand-in for the paper's variable-viscosity test)."""
    if contrast is not None:
        return 1.0 + (contrast - 1.0) * (1.0 - np.cos(2 * np.pi * x[..., 0])) / 2.0
    return 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])


# ---------------------------------------------------------------- quadrature grid

class Grid:
    """Tensor Gauss grid (p+2 points per element per direction) with the
    geometry and viscosity at every point; axis d of the arrays is direction d+1."""

    def __init__(self, S, amp=AMP, nu_const=None, npts=None, contrast=None, geometry_kind="sine_bump"):
        self.S = S
        self.kind = geometry_kind
        if geometry_kind == "annulus" and contrast is None and nu_const is None:
            nu_const = 1.0
        npts = S.p + 2 if npts is None else npts
        self.pts, self.wts = [], []
        for d in range(3):
            x, w = splines.gauss_rule(S.pres[d].knots, npts)
            self.pts.append(x)
            self.wts.append(w)
        self.amp, self.nu_const, self.contrast = amp, nu_const, contrast
        E = np.stack(np.meshgrid(*self.pts, indexing="ij"), axis=-1)
        self.x, self.J, self.det, self.Jinv = geometry(E, amp, geometry_kind)
        self.nu = self.nu_of(self.x)
        W = self.wts[0][:, None, None] * self.wts[1][None, :, None] * self.wts[2][None, None, :]
        self.W = W
        # univariate tables at the points: value and derivative of each space
        self.vtab = {}

    @property
    def identity(self):
        """True when the map is the identity (sine bump of amplitude 0)."""
        return self.kind == "sine_bump" and self.amp == 0.0

    def nu_of(self, x):
        """The viscosity at physical points x (..., 3)."""
        if self.nu_const is not None:
            return np.full(x.shape[:-1], float(self.nu_const))
        return viscosity(x, self.contrast)

    def at(self, E):
        """Geometry and viscosity at other parametric points E (..., 3), with the
        attributes J, det, Jinv, nu that the coefficient functions read."""
        P = _Points()
        P.x, P.J, P.det, P.Jinv = geometry(E, self.amp, self.kind)
        P.nu = self.nu_of(P.x)
        return P

    def face(self, d, t):
        """Parametric points (tensor grid, extent 1 along direction d) and face
        weights (product of the Gauss weights of the two other directions) of
        the face eta_d = t."""
        axes = [np.array([float(t)]) if e == d else self.pts[e] for e in range(3)]
        E = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
        w = [np.ones(1) if e == d else self.wts[e] for e in range(3)]
        W = w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
        return E, W

    def table(self, space, d, deriv):
        key = (id(space), d, deriv)
        if key not in self.vtab:
            B, D = splines.basis(space.knots, space.degree, self.pts[d])
            self.vtab[key] = ((D if deriv else B)[:, space.keep]).T.copy()   # (n, npts)
        return self.vtab[key]


class _Points:
    """Geometry and viscosity at a set of parametric points (see Grid.at)."""


def tables(G, space3, derivs, face=None):
    """Per-direction tables (n_d, q_d) of the basis (derivs[d] False) or its
    derivative; on a face (d, t) the direction-d table is the basis at eta_d = t."""
    T = []
    for e in range(3):
        s = space3[e]
        if face is not None and face[0] == e:
            B, D = splines.basis(s.knots, s.degree, np.array([float(face[1])]))
            T.append(((D if derivs[e] else B)[:, s.keep]).T.copy())
        else:
            T.append(G.table(s, e, derivs[e]))
    return T


def eval_tables(T, x):
    """sum_i x_i prod_d T_d[i_d, q_d], indexed [q1, q2, q3]; x vec-ordered (i1 fastest)."""
    n = [t.shape[0] for t in T]
    X = np.asarray(x, float).reshape(n[2], n[1], n[0])
    Y = np.einsum("cba,ap->cbp", X, T[0])
    Y = np.einsum("cbp,bq->cpq", Y, T[1])
    return np.einsum("cpq,cr->pqr", Y, T[2])


def test_tables(T, F):
    """Transpose of eval_tables: y_i = sum_q F[q] prod_d T_d[i_d, q_d] (vec order)."""
    Y = np.einsum("pqr,cr->pqc", F, T[2])
    Y = np.einsum("pqc,bq->pbc", Y, T[1])
    Y = np.einsum("pbc,ap->abc", Y, T[0])
    return np.transpose(Y, (2, 1, 0)).reshape(-1)


def to_points(G, space3, x, derivs):
    """Evaluate sum_i x_i prod_d T_d[i_d, q_d] where T_d is the value table of
    direction d (or its derivative when derivs[d]); x vec-ordered (i1 fastest)."""
    n = [space3[d].n for d in range(3)]
    X = np.asarray(x, float).reshape(n[2], n[1], n[0])        # [i3, i2, i1]
    T = [G.table(space3[d], d, derivs[d]) for d in range(3)]  # (n_d, q_d)
    # result indexed [q1, q2, q3]
    Y = np.einsum("cba,ap->cbp", X, T[0])
    Y = np.einsum("cbp,bq->cpq", Y, T[1])
    Y = np.einsum("cpq,cr->pqr", Y, T[2])
    return Y


def from_points(G, space3, F, derivs):
    """Transpose of to_points: y_i = sum_q F[q] prod_d T_d[i_d, q_d] (vec order)."""
    T = [G.table(space3[d], d, derivs[d]) for d in range(3)]
    Y = np.einsum("pqr,cr->pqc", F, T[2])
    Y = np.einsum("pqc,bq->pbc", Y, T[1])
    Y = np.einsum("pbc,ap->abc", Y, T[0])                      # [i1, i2, i3]
    return np.transpose(Y, (2, 1, 0)).reshape(-1)


# ---------------------------------------------------------------- mapped Stokes operator

def matvec(S, G, x):
    """y = A x on the mapped domain by sum-factorized quadrature: u and grad_eta u
    at the points, grad_x u = grad_eta u J^{-1}, stress 2 nu grad^s u - p I, tested
    with grad_x of the basis (a(.,.) and b(.,.) of Sec. 3)."""
    blocks = S.split(np.asarray(x, float))
    u, pr = blocks[:3], blocks[3]
    wd = G.W * G.det
    # grad_x u: gx[r][c] = d u_r / d x_c = sum_a d u_r/d eta_a (J^{-1})_{a c}
    gx = [[None] * 3 for _ in range(3)]
    for r in range(3):
        ge = [to_points(G, S.vel[r], u[r], [a == 0, a == 1, a == 2]) for a in range(3)]
        for c in range(3):
            gx[r][c] = sum(ge[a] * G.Jinv[..., a, c] for a in range(3))
    ph = to_points(G, S.pres, pr, [False, False, False])
    div = gx[0][0] + gx[1][1] + gx[2][2]
    ys = []
    for r in range(3):
        y = np.zeros(S.block_sizes[r])
        for a in range(3):
            # F_a = sum_c sigma_rc (J^{-1})_{a c}, sigma = nu (grad u + grad u^T) - p I
            Fa = np.zeros_like(G.det)
            for c in range(3):
                sig = G.nu * (gx[r][c] + gx[c][r]) - (ph if r == c else 0.0)
                Fa = Fa + sig * G.Jinv[..., a, c]
            y += from_points(G, S.vel[r], Fa * wd, [a == 0, a == 1, a == 2])
        ys.append(y)
    ys.append(from_points(G, S.pres, -div * wd, [False, False, False]))
    return np.concatenate(ys)


def brute_force(S, G):
    """Dense A (velocity) and B by explicit quadrature of 2 nu grad^s w : grad^s v
    and -q div v, every vector basis function evaluated on its own (tiny sizes)."""
    P = np.stack(np.meshgrid(np.arange(len(G.pts[0])), np.arange(len(G.pts[1])), np.arange(len(G.pts[2])),
                             indexing="ij"), axis=-1).reshape(-1, 3)
    Jinv = G.Jinv.reshape(-1, 3, 3)
    wd = (G.W * G.det).reshape(-1)
    nu = G.nu.reshape(-1)

    def multi(space3):
        n = [space3[d].n for d in range(3)]
        idx = np.array(np.unravel_index(np.arange(int(np.prod(n))), n[::-1])).T[:, ::-1]
        return idx

    def grad_x(space3, m):
        ge = np.ones((len(P), 3))
        for a in range(3):
            v = np.ones(len(P))
            for d in range(3):
                T = G.table(space3[d], d, d == a)
                v = v * T[m[d], P[:, d]]
            ge[:, a] = v
        return np.einsum("qa,qac->qc", ge, Jinv)       # d B / d x_c

    idx = multi(S.vel[0])
    nv = len(idx)
    grads = np.array([grad_x(S.vel[0], m) for m in idx])          # (nv, q, 3)
    A = np.zeros((3 * nv, 3 * nv))
    for r in range(3):
        for s in range(3):
            for i in range(nv):
                Gw = np.zeros((len(P), 3, 3))
                Gw[:, r, :] = grads[i]
                Sw = 0.5 * (Gw + Gw.transpose(0, 2, 1))
                for j in range(nv):
                    Gv = np.zeros((len(P), 3, 3))
                    Gv[:, s, :] = grads[j]
                    Sv = 0.5 * (Gv + Gv.transpose(0, 2, 1))
                    A[r * nv + i, s * nv + j] = np.sum(wd * 2 * nu * np.einsum("qab,qab->q", Sw, Sv))
    pidx = multi(S.pres)
    pval = np.array([np.prod([G.table(S.pres[d], d, False)[m[d], P[:, d]] for d in range(3)], axis=0)
                     for m in pidx])
    B = np.zeros((len(pidx), 3 * nv))
    for r in range(3):
        for j in range(nv):
            B[:, r * nv + j] = -(pval * grads[j][:, r][None, :]) @ wd
    return A, B


# ---------------------------------------------------------------- RT on the identity map: the Nitsche faces

def _nitsche_constants(S):
    """C_pen and, per direction d, the h of the penalty C_pen/h on the faces
    normal to e_d: the Nitsche factor of that direction (the same reading as
    the Kronecker form's K~_d)."""
    cp = {s.cpen for row in S.vel for s in row if s.nitsche}
    assert len(cp) == 1, cp
    hs = []
    for d in range(S.dim):
        hd = {S.vel[k][d].h for k in range(S.dim) if S.vel[k][d].nitsche}
        assert len(hd) == 1, hd
        hs.append(hd.pop())
    return cp.pop(), hs


def _require_rt_identity(S, G):
    if S.disc != "RT":
        raise ValueError("not a Raviart-Thomas system")
    if not G.identity:
        raise ValueError("the RT system is built on the identity map (no Piola push-forward)")


def nitsche_matvec(S, G, x):
    """The velocity blocks of sigma(u, .) (eq. theta) on the six faces of the
    cube, viscosity nu(x) at the face points, the RT basis e_k B on the identity
    map. Written from the form: with n the outward normal (-e_d on eta_d = 0,
    +e_d on eta_d = 1) and v = e_s B_j the test function,
        2 nu [C_pen/h u.v - ((grad^s u) n).v - ((grad^s v) n).u]
    (h = the element size along d, the penalty of the direction-d factor K~_d)
    where ((grad^s v) n).u = (u_s d_n B_j + (u.n) d_s B_j) / 2. Face quadrature:
    the volume rule's points of the two other directions."""
    _require_rt_identity(S, G)
    cpen, h = _nitsche_constants(S)
    u = S.split(np.asarray(x, float))[:3]
    ys = [np.zeros(S.block_sizes[k]) for k in range(3)]
    unit = [[e == b for e in range(3)] for b in range(3)]
    for d in range(3):
        for t, sgn in ((0.0, -1.0), (1.0, 1.0)):
            face = (d, t)
            E, Wf = G.face(d, t)
            w2 = 2.0 * G.at(E).nu * Wf
            val = [eval_tables(tables(G, S.vel[c], [False] * 3, face), u[c]) for c in range(3)]
            grd = [[eval_tables(tables(G, S.vel[c], unit[b], face), u[c]) for b in range(3)] for c in range(3)]
            # ((grad^s u) n)_a = (d_d u_a + d_a u_d) sgn / 2
            sn = [0.5 * sgn * (grd[a][d] + grd[d][a]) for a in range(3)]
            for s_ in range(3):
                ys[s_] += test_tables(tables(G, S.vel[s_], [False] * 3, face), w2 * (cpen / h[d] * val[s_] - sn[s_]))
                ys[s_] += test_tables(tables(G, S.vel[s_], unit[d], face), -0.5 * sgn * w2 * val[s_])
                ys[s_] += test_tables(tables(G, S.vel[s_], unit[s_], face), -0.5 * sgn * w2 * val[d])
    return ys


def operator(S, G, x):
    """A x: the volume forms (matvec) and, for RT, the Nitsche form sigma."""
    y = matvec(S, G, x)
    if S.disc == "RT":
        nv = sum(S.block_sizes[:3])
        y[:nv] += np.concatenate(nitsche_matvec(S, G, x))
    return y


def nitsche_diag(S, G, k):
    """diag of the sigma part of A_kk: sum over faces of
    int 2 nu [C_pen/h B_i^2 - 2 ((grad^s e_k B_i) n)_k B_i], with
    ((grad^s e_k B) n)_k = (d_n B + n_k d_k B) / 2."""
    _require_rt_identity(S, G)
    cpen, h = _nitsche_constants(S)
    out = np.zeros(S.block_sizes[k])
    sp = S.vel[k]
    for d in range(3):
        for t, sgn in ((0.0, -1.0), (1.0, 1.0)):
            face = (d, t)
            E, Wf = G.face(d, t)
            w2 = 2.0 * G.at(E).nu * Wf
            V = tables(G, sp, [False] * 3, face)
            D = tables(G, sp, [e == d for e in range(3)], face)
            sq = [V[e] * V[e] for e in range(3)]
            mixed_d = [V[e] * (D[e] if e == d else V[e]) for e in range(3)]
            factor = sgn * (2.0 if d == k else 1.0)        # d_n B + n_k d_k B = sgn (1 + delta_dk) d_d B
            out += cpen / h[d] * test_tables(sq, w2) - factor * test_tables(mixed_d, w2)
    return out


# ---------------------------------------------------------------- coefficients and separable fit

def c_diag(G, k):
    """c^k_jj = nu |det J| ((J^{-1} J^{-T})_jj + (J^{-1})_jk^2), j = 0..2 (eq. Q_TH)."""
    Ji = G.Jinv
    JJt = np.einsum("...ac,...bc->...ab", Ji, Ji)
    return [G.nu * np.abs(G.det) * (JJt[..., j, j] + Ji[..., j, k] ** 2) for j in range(3)]


def c_matrix_rt(J, det, Jinv, nu, k):
    """C_k^RT = nu |det J| J^{-1} (||R_k||^2 I + R_k R_k^T) J^{-T} with R_k = J e_k / det J (eq. Q_RT)."""
    R = J[..., :, k] / det[..., None]
    M = (R * R).sum(-1)[..., None, None] * np.eye(3) + R[..., :, None] * R[..., None, :]
    C = np.einsum("...ab,...bc,...dc->...ad", Jinv, M, Jinv)
    return (nu * np.abs(det))[..., None, None] * C


def c_diag_rt(G, k):
    """c^k_jj of C_k^RT (eq. Q_RT), j = 0..2."""
    C = c_matrix_rt(G.J, G.det, G.Jinv, G.nu, k)
    return [C[..., j, j] for j in range(3)]


def separable_fit(c, sweeps=SWEEPS):
    """log c ~ f1(q1) + f2(q2) + f3(q3) by Diliberto-Straus midrange sweeps."""
    L = np.log(c)
    f = [np.zeros(L.shape[d]) for d in range(3)]
    shp = [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]
    for _ in range(sweeps):
        for d in range(3):
            R = L - sum(f[e].reshape(shp[e]) for e in range(3) if e != d)
            axes = tuple(e for e in range(3) if e != d)
            f[d] = 0.5 * (R.max(axis=axes) + R.min(axis=axes))
    return f


def fit_at(L_face, f, d):
    """The direction-d factor of a converged fit log c ~ f_1 + f_2 + f_3 at a
    point outside the grid (a face eta_d = t): the fit's own update for
    direction d, the midrange over the face of log c - sum_{e != d} f_e
    (L_face has extent 1 along d)."""
    shp = [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]
    R = L_face - sum(f[e].reshape(shp[e]) for e in range(3) if e != d)
    return 0.5 * (R.max() + R.min())


def tau_mu(G, k, sweeps=SWEEPS, disc="TH"):
    """tau^k_d and mu^k_d at the quadrature points of direction d (Appendix form);
    for RT also tau^k_d at eta_d = 0 and 1 (the boundary terms of the weighted
    K~), returned as a third list of pairs. Reading: the fit is computed on the
    quadrature points as the Appendix says, and its direction-d factor is
    carried to the faces by the fit's own update there (fit_at), so that the
    interior fit is unchanged."""
    cfun = c_diag_rt if disc == "RT" else c_diag
    cs = cfun(G, k)
    fits = []
    for j in range(3):
        f = separable_fit(cs[j], sweeps)
        # normalize: non-own factors with zero mean log, constant into the own factor
        for e in range(3):
            if e != j:
                m = f[e].mean()
                f[e] = f[e] - m
                f[j] = f[j] + m
        fits.append(f)
    tau = [np.exp(fits[d][d]) for d in range(3)]
    mu = [np.exp(0.5 * sum(fits[j][d] for j in range(3) if j != d)) for d in range(3)]
    if disc != "RT":
        return tau, mu
    ends = []
    for d in range(3):
        pair = []
        for t in (0.0, 1.0):
            E, _ = G.face(d, t)
            L = np.log(cfun(G.at(E), k)[d])
            pair.append(float(np.exp(fit_at(L, fits[d], d))))
        ends.append(tuple(pair))
    return tau, mu, ends


def weighted_pencils(S, G, k, sweeps=SWEEPS):
    """(K^k_d, M^k_d) with weights tau^k_d, mu^k_d given at the quadrature points;
    for RT the tangential factors are the weighted K~, M~ of the Appendix, the
    Nitsche boundary terms scaled by tau^k_d(0) and tau^k_d(1)."""
    if S.disc == "RT":
        _require_rt_identity(S, G)
        tau, mu, ends = tau_mu(G, k, sweeps, "RT")
    else:
        tau, mu = tau_mu(G, k, sweeps)
    Ks, Ms = [], []
    for d in range(3):
        sp = S.vel[k][d]
        Tv = G.table(sp, d, False)
        Td = G.table(sp, d, True)
        w = G.wts[d]
        K = (Td * (w * tau[d])) @ Td.T
        if sp.nitsche:
            K = K - uv.nitsche_boundary(sp, ends[d][0], ends[d][1])
        Ks.append(K)
        Ms.append((Tv * (w * mu[d])) @ Tv.T)
    return Ks, Ms


# ---------------------------------------------------------------- diagonals and P_D^G

def diag_A(S, G, k):
    """[A_kk]_ii = sum_ab int C^kk_ab d_a B_i d_b B_i with C^kk = nu |J| (J^-1 J^-T + D_k D_k^T)."""
    Ji = G.Jinv
    C = G.nu[..., None, None] * np.abs(G.det)[..., None, None] * (
        np.einsum("...ac,...bc->...ab", Ji, Ji) + Ji[..., :, k][..., :, None] * Ji[..., :, k][..., None, :])
    out = 0.0
    for a in range(3):
        for b in range(3):
            T = []
            for d in range(3):
                Ta = G.table(S.vel[k][d], d, d == a)
                Tb = G.table(S.vel[k][d], d, d == b)
                T.append(Ta * Tb)
            F = C[..., a, b] * G.W
            Y = np.einsum("pqr,cr->pqc", F, T[2])
            Y = np.einsum("pqc,bq->pbc", Y, T[1])
            Y = np.einsum("pbc,ap->abc", Y, T[0])
            out = out + np.transpose(Y, (2, 1, 0)).reshape(-1)
    return out


def diag_Q(S, G):
    """[Q]_ii = int nu^{-1} g B_i^2 with g = |det J| (TH) or |det J|^{-1} (RT)
    (eq. weighted-pressure-mass)."""
    T = [G.table(S.pres[d], d, False) ** 2 for d in range(3)]
    g = np.abs(G.det) if S.disc != "RT" else 1.0 / np.abs(G.det)
    F = G.W * g / G.nu
    Y = np.einsum("pqr,cr->pqc", F, T[2])
    Y = np.einsum("pqc,bq->pbc", Y, T[1])
    Y = np.einsum("pbc,ap->abc", Y, T[0])
    return np.transpose(Y, (2, 1, 0)).reshape(-1)


def kron_diag(factors):
    """diag(A_3 x A_2 x A_1) in vec order."""
    d = np.ones(1)
    for A in reversed(factors):
        d = np.kron(d, np.diag(A))
    return d


class PDG:
    """The geometry-aware block preconditioner P_D^G = diag(P_V^G, P_Q^G)."""

    def __init__(self, S, G, sweeps=SWEEPS):
        self.S = S
        self.pencils, self.DV = [], []
        for k in range(3):
            Ks, Ms = weighted_pencils(S, G, k, sweeps)
            self.pencils.append((Ks, Ms, [1.0, 1.0, 1.0]))
            dP = sum(kron_diag([Ks[e] if e == d else Ms[e] for e in range(3)]) for d in range(3))
            dA = diag_A(S, G, k)
            if S.disc == "RT":
                dA = dA + nitsche_diag(S, G, k)
            self.DV.append(dA / dP)
        self.Mp = stokes.pq_factors(S)
        self.DQ = diag_Q(S, G) / kron_diag(self.Mp)

    def apply(self, r):
        b = self.S.split(np.asarray(r, float))
        return np.concatenate(self.apply_v(b[:3]) + [self.apply_q(b[3])])

    def apply_v(self, blocks):
        """(P_V^G)^{-1} on the three velocity blocks."""
        out = []
        for k in range(3):
            Ks, Ms, coef = self.pencils[k]
            sc = self.DV[k] ** -0.5
            out.append(sc * kron.fd_solve(Ks, Ms, coef, sc * blocks[k]))
        return out

    def apply_q(self, rq):
        """(P_Q^G)^{-1} on the pressure block."""
        sq = self.DQ ** -0.5
        return sq * kron.kron_mass_solve(self.Mp, sq * rq)


def coupling(S, G, u_blocks=None, q=None):
    """B u (pressure block) or B^T q (velocity blocks) on the mapped domain: the
    off-diagonal blocks of the operator, read off the matvec with the other
    unknowns zero."""
    z = [np.zeros(n) for n in S.block_sizes]
    if q is not None:
        z[3] = q
        return S.split(matvec(S, G, np.concatenate(z)))[:3]
    z[:3] = u_blocks
    return S.split(matvec(S, G, np.concatenate(z)))[3]


def apply_PTG_inv(S, G, pdg, r):
    """P_T^G = [[P_V^G, B^T], [0, -P_Q^G]] (Sec. 6, eq. P_T with the geometry-aware
    blocks): q = -(P_Q^G)^{-1} r_q, u = (P_V^G)^{-1} (r_u - B^T q)."""
    b = S.split(np.asarray(r, float))
    q = -pdg.apply_q(b[3])
    bt = coupling(S, G, q=q)
    u = pdg.apply_v([b[k] - bt[k] for k in range(3)])
    return np.concatenate(u + [q])


def apply_PCG_inv(S, G, pdg, r):
    """P_C^G by the product form of its inverse (Sec. 4) with the geometry-aware blocks."""
    b = S.split(np.asarray(r, float))
    z = pdg.apply_v(b[:3])
    q = -pdg.apply_q(b[3] - coupling(S, G, u_blocks=z))
    w = pdg.apply_v(coupling(S, G, q=q))
    return np.concatenate([z[k] - w[k] for k in range(3)] + [q])


def operator_row(S, G, blk, i_multi):
    """All nonzero entries of one row of the mapped operator, by quadrature of the
    definitions at the points of the row function's support (sampled checks at
    full size): velocity row blk < 3 (function e_blk B_i) against every velocity
    and pressure function, pressure row blk == 3 against every velocity function.
    Returns {global column index: value}."""
    off = np.concatenate([[0], np.cumsum(S.block_sizes)])
    row_space = S.vel[blk] if blk < 3 else S.pres
    # support points of the row function in each direction
    sup = []
    for d in range(3):
        T = G.table(row_space[d], d, False)
        Td = G.table(row_space[d], d, True)
        nz = np.nonzero((np.abs(T[i_multi[d]]) + np.abs(Td[i_multi[d]])) > 0)[0]
        sup.append(nz)
    ix = np.ix_(sup[0], sup[1], sup[2])
    Jinv = G.Jinv[ix]
    wd = (G.W * G.det)[ix]
    nu = G.nu[ix]

    def fields(space3, m, deriv_dir):
        v = 1.0
        for d in range(3):
            T = G.table(space3[d], d, deriv_dir == d)[m[d]][sup[d]]
            sh = [1, 1, 1]
            sh[d] = -1
            v = v * T.reshape(sh)
        return v

    def grad_x(space3, m):
        ge = np.stack([fields(space3, m, a) for a in range(3)], axis=-1)
        return np.einsum("...a,...ac->...c", ge, Jinv)

    def candidates(space3):
        out = []
        for d in range(3):
            T = G.table(space3[d], d, False)
            Td = G.table(space3[d], d, True)
            act = np.nonzero(((np.abs(T[:, sup[d]]) + np.abs(Td[:, sup[d]])) > 0).any(axis=1))[0]
            out.append(act)
        return out

    res = {}
    if blk < 3:
        gi = grad_x(S.vel[blk], i_multi)
        for s in range(3):
            c = candidates(S.vel[s])
            for j3 in c[2]:
                for j2 in c[1]:
                    for j1 in c[0]:
                        gj = grad_x(S.vel[s], (j1, j2, j3))
                        # 2 nu grad^s(e_blk B_i) : grad^s(e_s B_j) = nu (delta gi.gj + d_s B_i d_blk B_j)
                        Gw = np.zeros(gi.shape[:-1] + (3, 3))
                        Gw[..., blk, :] = gi
                        Gv = np.zeros(gi.shape[:-1] + (3, 3))
                        Gv[..., s, :] = gj
                        Sw = 0.5 * (Gw + np.swapaxes(Gw, -1, -2))
                        Sv = 0.5 * (Gv + np.swapaxes(Gv, -1, -2))
                        v = np.sum(wd * 2 * nu * np.einsum("...ab,...ab->...", Sw, Sv))
                        col = off[s] + (j3 * S.vel[s][1].n + j2) * S.vel[s][0].n + j1
                        res[int(col)] = v
        c = candidates(S.pres)
        for l3 in c[2]:
            for l2 in c[1]:
                for l1 in c[0]:
                    v = -np.sum(wd * fields(S.pres, (l1, l2, l3), -1) * gi[..., blk])
                    col = off[3] + (l3 * S.pres[1].n + l2) * S.pres[0].n + l1
                    res[int(col)] = v
    else:
        rho = fields(S.pres, i_multi, -1)
        for r in range(3):
            c = candidates(S.vel[r])
            for j3 in c[2]:
                for j2 in c[1]:
                    for j1 in c[0]:
                        gj = grad_x(S.vel[r], (j1, j2, j3))
                        v = -np.sum(wd * rho * gj[..., r])
                        col = off[r] + (j3 * S.vel[r][1].n + j2) * S.vel[r][0].n + j1
                        res[int(col)] = v
    return res
