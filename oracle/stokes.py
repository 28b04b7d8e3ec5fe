"""Isogeometric Stokes system on the unit square / cube and its block
preconditioner (paper Sec. 2.2, Sec. 3, Sec. 4, Sec. 5). Oracle: test
infrastructure only.

Unknown ordering (Sec. 3, eq. Stokes_system): [u_1; u_2; (u_3;) p], every block
vec-ordered with i1 fastest; velocity basis indices are the interior ones for
Taylor-Hood (eq. V_TH_0_basis1) and the normal-interior ones for
Raviart-Thomas (eq. basisRT_V1).

Identity map, constant viscosity nu (Sec. 7, cube; L^2 forms of eq. a_form):
  [A_rs]_{ij} = nu int (delta_rs grad B_i . grad B_j + d_s B_i d_r B_j)
  [B_r]_{lj}  = - int rho_l d_r B_j
(from 2 nu grad^s w : grad^s v with w = e_r B_i, v = e_s B_j), so that
A_kk = P_{V,k} (Sec. 7, "A_kk = P_V,k" on the cube) and every block is one or
a few Kronecker products of univariate mixed matrices. The RT Nitsche form
sigma adds only to A_kk on the cube (its cross terms vanish because a
component vanishes together with its tangential derivatives on the faces
normal to it).

Pins (tests/test_oracle_stokes.py): Kronecker blocks vs. brute-force
element quadrature of a(.,.) and b(.,.) written from the symmetric-gradient
definition (TH), and for RT of a(.,.) + sigma(.,.) (the Nitsche form of
eq. theta, face by face with outward normals) and b(.,.), all blocks A_rs
including r != s, which pins the reading that sigma adds only to A_kk on the
cube; A_kk = P_{V,k}; B^T 1 = 0 (constant pressure in the kernel); symmetry
of the assembled operator; P_V, P_Q SPD.
"""
from dataclasses import dataclass

import numpy as np

from . import kron, splines, univariate as uv


@dataclass
class Stokes:
    dim: int
    disc: str            # "TH" or "RT"
    p: int               # pressure degree
    vel: list            # vel[k][d]: Space1D of velocity component k in direction d
    pres: list           # pres[d]:   Space1D of the pressure in direction d
    nu: float = 1.0

    @property
    def vel_shapes(self):
        return [tuple(s.n for s in self.vel[k]) for k in range(self.dim)]

    @property
    def pres_shape(self):
        return tuple(s.n for s in self.pres)

    @property
    def block_sizes(self):
        return [int(np.prod(s)) for s in self.vel_shapes] + [int(np.prod(self.pres_shape))]

    @property
    def n_total(self):
        return int(sum(self.block_sizes))

    def split(self, x):
        out, o = [], 0
        for n in self.block_sizes:
            out.append(x[o:o + n])
            o += n
        return out


def build(pressure_knots, p, disc="TH", cpen=None, nu=1.0, velocity="th"):
    """Spaces of Sec. 2.2 from the pressure knot vector of each direction.
    TH: velocity = degree p+1 with the same regularity (Sec. 2.2.1), interior indices;
    velocity="max_smooth" instead keeps every interior breakpoint simple (degree p+1,
    C^p: only the end knots gain a copy), the maximal-smoothness space that an
    "about 68^3 velocity unknowns" count at 64^3 elements, p = 3 corresponds to.
    RT: component k has degree p+1 and one more continuity in direction k, end
    functions removed there; degree p and all functions elsewhere, with the
    Nitsche terms, C_pen = 5(alpha+1) (Sec. 7) and h = the largest knot span."""
    dim = len(pressure_knots)
    pres = [uv.full_space(np.asarray(t, float), p) for t in pressure_knots]
    vel = []
    for k in range(dim):
        row = []
        for d in range(dim):
            t = np.asarray(pressure_knots[d], float)
            if disc == "TH" and velocity == "max_smooth":
                row.append(uv.interior_space(np.concatenate([[0.0], t, [1.0]]), p + 1))
            elif disc == "TH":
                row.append(uv.interior_space(splines.elevate_knots(t, p), p + 1))
            elif disc == "RT":
                if d == k:
                    tk = np.concatenate([[0.0], t, [1.0]])   # degree p+1, same multiplicities
                    row.append(uv.interior_space(tk, p + 1))
                else:
                    z = splines.breakpoints(t)
                    h = float(np.max(np.diff(z)))
                    inner_mult = int(np.sum(t == z[1])) if len(z) > 2 else 1
                    alpha = p - inner_mult
                    c = 5.0 * (alpha + 1) if cpen is None else cpen
                    row.append(uv.full_space(t, p, nitsche=True, cpen=c, h=h))
            else:
                raise ValueError(disc)
        vel.append(row)
    return Stokes(dim, disc, p, vel, pres, nu)


def build_uniform(n_el, p, dim, disc="TH", regularity=None, cpen=None, nu=1.0, velocity="th"):
    alpha = p - 1 if regularity is None else regularity
    n = [n_el] * dim if np.isscalar(n_el) else list(n_el)
    knots = [splines.open_knots(n[d], p, alpha) for d in range(dim)]
    return build(knots, p, disc, cpen, nu, velocity)


# ---------------------------------------------------------------- preconditioner

def pv_pencils(S, k):
    """Univariate (K_d, M_d) of P_{V,k} and the coefficients c_{k,d} = 1 + delta_dk
    (eq. prec3D_TH / prec3D_RT; reading for 2D: drop direction 3)."""
    Ks = [uv.stiffness(s) for s in S.vel[k]]
    Ms = [uv.mass(s) for s in S.vel[k]]
    coef = [2.0 if d == k else 1.0 for d in range(S.dim)]
    return Ks, Ms, coef


def pq_factors(S):
    """P_Q = M_3 (x) M_2 (x) M_1, pressure mass matrices (eq. precQ)."""
    return [uv.mass(s) for s in S.pres]


def pv_matrix(S, k):
    return kron.kron_sum_matrix(*pv_pencils(S, k))


def apply_PD_inv(S, r, method="fd"):
    """s = P_D^{-1} r, P_D = diag(P_V, P_Q) (eq. P_D). method "fd" uses
    Algorithm 1 for P_V and banded solves for P_Q; "dense" uses dense LU."""
    blocks = S.split(np.asarray(r, float))
    out = []
    for k in range(S.dim):
        Ks, Ms, coef = pv_pencils(S, k)
        if method == "fd":
            out.append(kron.fd_solve(Ks, Ms, coef, blocks[k]))
        else:
            out.append(kron.dense_solve(Ks, Ms, coef, blocks[k]))
    Mp = pq_factors(S)
    if method == "fd":
        out.append(kron.kron_mass_solve(Mp, blocks[-1]))
    else:
        out.append(np.linalg.solve(kron.kron_matrix(Mp), blocks[-1]))
    return np.concatenate(out)


# ---------------------------------------------------------------- operator

def a_block_terms(S, r, s):
    """Kronecker terms (coef, factors in mode order) of A_rs on the identity map."""
    if r == s:
        Ks, Ms, coef = pv_pencils(S, r)
        return [(S.nu * c, f) for c, f in kron.kron_sum_terms(Ks, Ms, coef)]
    f = []
    for d in range(S.dim):
        if d == s:
            f.append(uv.mixed(S.vel[r][d], 1, S.vel[s][d], 0))
        elif d == r:
            f.append(uv.mixed(S.vel[r][d], 0, S.vel[s][d], 1))
        else:
            f.append(uv.mixed(S.vel[r][d], 0, S.vel[s][d], 0))
    return [(S.nu, f)]


def b_block_terms(S, r):
    """B_r = - (x)_d (int rho b^(delta_dr)), rows pressure, cols velocity comp. r."""
    f = [uv.mixed(S.pres[d], 0, S.vel[r][d], 1 if d == r else 0) for d in range(S.dim)]
    return [(-1.0, f)]


def _apply_terms(terms, x):
    return sum(c * kron.kron_apply(f, x) for c, f in terms)


def _apply_terms_T(terms, x):
    return sum(c * kron.kron_apply([A.T for A in f], x) for c, f in terms)


def matvec(S, x):
    """y = A x for the block system of eq. Stokes_system (matrix-free Kronecker form)."""
    blocks = S.split(np.asarray(x, float))
    u, pr = blocks[:S.dim], blocks[-1]
    ys = []
    for r in range(S.dim):
        y = np.zeros(S.block_sizes[r])
        for s in range(S.dim):
            y += _apply_terms(a_block_terms(S, r, s), u[s])
        y += _apply_terms_T(b_block_terms(S, r), pr)
        ys.append(y)
    yp = np.zeros(S.block_sizes[-1])
    for r in range(S.dim):
        yp += _apply_terms(b_block_terms(S, r), u[r])
    ys.append(yp)
    return np.concatenate(ys)


def assembled(S):
    """Dense system matrix (tiny sizes only)."""
    d = S.dim
    nb = S.block_sizes
    off = np.concatenate([[0], np.cumsum(nb)])
    A = np.zeros((off[-1], off[-1]))
    for r in range(d):
        for s in range(d):
            A[off[r]:off[r + 1], off[s]:off[s + 1]] = sum(c * kron.kron_matrix(f) for c, f in a_block_terms(S, r, s))
        Br = sum(c * kron.kron_matrix(f) for c, f in b_block_terms(S, r))
        A[off[d]:, off[r]:off[r + 1]] = Br
        A[off[r]:off[r + 1], off[d]:] = Br.T
    return A


# ---------------------------------------------------------------- brute force

def apply_B(S, u_blocks):
    """B u (pressure block) for velocity blocks u_k (eq. Stokes_system)."""
    return sum(_apply_terms(b_block_terms(S, r), u_blocks[r]) for r in range(S.dim))


def apply_Bt(S, q):
    """B^T q (velocity blocks) for a pressure block q."""
    return [_apply_terms_T(b_block_terms(S, r), q) for r in range(S.dim)]


def _pv_solve(S, blocks, method):
    out = []
    for k in range(S.dim):
        Ks, Ms, coef = pv_pencils(S, k)
        out.append(kron.fd_solve(Ks, Ms, coef, blocks[k]) if method == "fd"
                   else kron.dense_solve(Ks, Ms, coef, blocks[k]))
    return out


def _pq_solve(S, rq, method):
    Mp = pq_factors(S)
    return kron.kron_mass_solve(Mp, rq) if method == "fd" else np.linalg.solve(kron.kron_matrix(Mp), rq)


def apply_PT_inv(S, r, method="fd"):
    """s = P_T^{-1} r for the block upper-triangular P_T = [[P_V, B^T], [0, -P_Q]]
    (eq. P_T): back substitution, q = -P_Q^{-1} r_q, then u = P_V^{-1} (r_u - B^T q)."""
    blocks = S.split(np.asarray(r, float))
    q = -_pq_solve(S, blocks[-1], method)
    bt = apply_Bt(S, q)
    u = _pv_solve(S, [blocks[k] - bt[k] for k in range(S.dim)], method)
    return np.concatenate(u + [q])


def apply_PC_inv(S, r, method="fd"):
    """s = P_C^{-1} r for P_C = [[P_V, B^T], [B, B P_V^{-1} B^T - P_Q]] (eq. P_C) by the
    paper's product form of its inverse, applied right to left: z = P_V^{-1} r_u;
    t = r_q - B z; q = -P_Q^{-1} t; u = z - P_V^{-1} B^T q."""
    blocks = S.split(np.asarray(r, float))
    z = _pv_solve(S, blocks[:S.dim], method)
    q = -_pq_solve(S, blocks[-1] - apply_B(S, z), method)
    w = _pv_solve(S, apply_Bt(S, q), method)
    return np.concatenate([z[k] - w[k] for k in range(S.dim)] + [q])


def pt_matrix(S):
    """Dense P_T (tiny sizes only)."""
    return _block_prec_matrix(S, lower=False)


def pc_matrix(S):
    """Dense P_C (tiny sizes only)."""
    return _block_prec_matrix(S, lower=True)


def _block_prec_matrix(S, lower):
    d = S.dim
    off = np.concatenate([[0], np.cumsum(S.block_sizes)])
    A = assembled(S)
    PV = np.zeros((off[d], off[d]))
    for k in range(d):
        PV[off[k]:off[k + 1], off[k]:off[k + 1]] = pv_matrix(S, k)
    PQ = kron.kron_matrix(pq_factors(S))
    Bt = A[:off[d], off[d]:]
    P = np.zeros_like(A)
    P[:off[d], :off[d]] = PV
    P[:off[d], off[d]:] = Bt
    P[off[d]:, off[d]:] = -PQ
    if lower:
        P[off[d]:, :off[d]] = Bt.T
        P[off[d]:, off[d]:] += Bt.T @ np.linalg.solve(PV, Bt)
    return P


def brute_force_TH(S, nu=1.0):
    """Dense A and B of the TH system by element-wise tensor Gauss quadrature of
    a(w,v) = int 2 nu grad^s w : grad^s v and b(v,q) = -int q div v, evaluating
    every vector basis function e_k B_i explicitly (tiny sizes only)."""
    assert S.disc == "TH"
    d = S.dim
    pts, wts = [], []
    for e in range(d):
        x, w = splines.gauss_rule(S.vel[0][e].knots, S.p + 2)
        pts.append(x)
        wts.append(w)
    grids = np.meshgrid(*pts, indexing="ij")       # axis e <-> direction e
    W = np.ones_like(grids[0])
    for e in range(d):
        sh = [1] * d
        sh[e] = -1
        W = W * wts[e].reshape(sh)
    W = W.reshape(-1)
    # univariate values at the points of each direction
    vb = []
    for e in range(d):
        B, D = splines.basis(S.vel[0][e].knots, S.vel[0][e].degree, pts[e])
        vb.append((B[:, S.vel[0][e].keep], D[:, S.vel[0][e].keep]))
    pb = []
    for e in range(d):
        B, _ = splines.basis(S.pres[e].knots, S.pres[e].degree, pts[e])
        pb.append(B[:, S.pres[e].keep])

    npt = [len(x) for x in pts]
    idx_v = np.array(np.unravel_index(np.arange(int(np.prod([vb[e][0].shape[1] for e in range(d)]))),
                                      [vb[e][0].shape[1] for e in reversed(range(d))])).T[:, ::-1]
    idx_p = np.array(np.unravel_index(np.arange(int(np.prod([pb[e].shape[1] for e in range(d)]))),
                                      [pb[e].shape[1] for e in reversed(range(d))])).T[:, ::-1]
    P = np.array(np.unravel_index(np.arange(int(np.prod(npt))), npt)).T    # point multi-index, dir 1 slowest

    def eval_vel(i_multi, deriv):
        v = np.ones(len(P))
        for e in range(d):
            T = vb[e][1] if deriv == e else vb[e][0]
            v = v * T[P[:, e], i_multi[e]]
        return v

    nv = len(idx_v)
    val = np.array([eval_vel(m, -1) for m in idx_v])                       # (nv, npts)
    grad = np.array([[eval_vel(m, e) for e in range(d)] for m in idx_v])   # (nv, d, npts)
    pval = np.array([np.prod([pb[e][P[:, e], m[e]] for e in range(d)], axis=0) for m in idx_p])

    A = np.zeros((d * nv, d * nv))
    Bm = np.zeros((len(idx_p), d * nv))
    for r in range(d):
        for s in range(d):
            # symmetric gradients of w = e_r B_i and v = e_s B_j at every point
            for i in range(nv):
                Gw = np.zeros((d, d, len(P)))
                Gw[r, :, :] = grad[i]
                Sw = 0.5 * (Gw + Gw.transpose(1, 0, 2))
                for j in range(nv):
                    Gv = np.zeros((d, d, len(P)))
                    Gv[s, :, :] = grad[j]
                    Sv = 0.5 * (Gv + Gv.transpose(1, 0, 2))
                    A[r * nv + i, s * nv + j] = np.sum(W * 2.0 * nu * np.einsum("abp,abp->p", Sw, Sv))
    for r in range(d):
        for j in range(nv):
            div = grad[j][r]          # div(e_r B_j) = d_r B_j
            Bm[:, r * nv + j] = -(pval * div[None, :]) @ W
    return A, Bm


def _tensor_points(rules, fixed=None):
    """Tensor-product points (N, d) and weights (N,) from per-direction rules;
    fixed = (e, t) pins coordinate e to t and drops its weight (a face)."""
    d = len(rules)
    axes, wts = [], []
    for e in range(d):
        if fixed is not None and fixed[0] == e:
            axes.append(np.array([float(fixed[1])]))
            wts.append(np.array([1.0]))
        else:
            axes.append(rules[e][0])
            wts.append(rules[e][1])
    grid = np.meshgrid(*axes, indexing="ij")
    W = np.ones_like(grid[0])
    for e in range(d):
        sh = [1] * d
        sh[e] = -1
        W = W * wts[e].reshape(sh)
    return np.stack([g.reshape(-1) for g in grid], axis=1), W.reshape(-1)


def _vector_basis(spaces, k, d, X):
    """Values (n, d, N) and gradients (n, d, d, N) of every vector basis
    function e_k B_i of component k at the points X, B_i the tensor product of
    the component's univariate spaces (index 1 fastest); [G]_{a,b} = d_b v_a."""
    vals, ders = [], []
    for e in range(d):
        s = spaces[e]
        B, D = splines.basis(s.knots, s.degree, X[:, e])
        vals.append(B[:, s.keep])
        ders.append(D[:, s.keep])
    shape = [vals[e].shape[1] for e in range(d)]
    n = int(np.prod(shape))
    multi = np.array(np.unravel_index(np.arange(n), shape[::-1])).T[:, ::-1]   # (n, d), index 1 fastest
    V = np.zeros((n, d, len(X)))
    G = np.zeros((n, d, d, len(X)))
    for f, m in enumerate(multi):
        V[f, k] = np.prod([vals[e][:, m[e]] for e in range(d)], axis=0)
        for b in range(d):
            G[f, k, b] = np.prod([(ders[e] if e == b else vals[e])[:, m[e]] for e in range(d)], axis=0)
    return V, G


def brute_force_RT(S, cpen, h, nu=1.0, faces=True):
    """Dense A (with the Nitsche form) and B of the RT system on the unit
    square / cube, written straight from the forms of Sec. 3 (eq. RT_dis):
      a(w, v)     = int_Omega 2 nu grad^s w : grad^s v,
      sigma(w, v) = int_dOmega 2 nu [C_pen/h w.v - ((grad^s w) n).v - ((grad^s v) n).w]   (eq. theta),
      b(v, q)     = - int_Omega q div v,
    with every vector basis function e_k B_i evaluated on its own, the volume
    integrals by tensor Gauss quadrature and the boundary integral face by
    face (outward unit normal -e_d on eta_d = 0 and +e_d on eta_d = 1) with
    the same rule on the face's own directions. Nothing here uses the
    univariate factors, so it pins the Kronecker blocks of A_rs for all r, s
    (the claim that sigma adds only to A_kk included). faces=False leaves
    sigma out (the volume form alone). nu is a constant or a function of the
    points (N, d) -> (N,) (a variable viscosity); h is one mesh size or one per
    direction (the faces normal to e_d take h[d]). Tiny sizes only."""
    assert S.disc == "RT"
    d = S.dim
    npts = S.p + 2
    rules = []
    for e in range(d):
        z = np.unique(np.concatenate([S.vel[k][e].knots for k in range(d)] + [S.pres[e].knots]))
        rules.append(splines.gauss_rule(z, npts))
    X, W = _tensor_points(rules)
    face_rules = []
    for e in range(d if faces else 0):
        for t, sgn in ((0.0, -1.0), (1.0, 1.0)):
            Xf, Wf = _tensor_points(rules, fixed=(e, t))
            nrm = np.zeros(d)
            nrm[e] = sgn
            face_rules.append((Xf, Wf, nrm, float(h[e]) if np.ndim(h) else float(h)))

    def all_vel(P):
        Vs, Gs = zip(*[_vector_basis(S.vel[k], k, d, P) for k in range(d)])
        V = np.concatenate(Vs)
        G = np.concatenate(Gs)
        return V, 0.5 * (G + G.transpose(0, 2, 1, 3)), G

    nu_at = nu if callable(nu) else (lambda P: np.full(len(P), float(nu)))
    V, Sg, G = all_vel(X)
    A = np.einsum("iabp,jabp,p->ij", Sg, Sg, 2.0 * nu_at(X) * W)
    for Xf, Wf, nrm, hf in face_rules:
        Vf, Sf, _ = all_vel(Xf)
        Sn = np.einsum("iabp,b->iap", Sf, nrm)                 # (grad^s v) n
        w2 = 2.0 * nu_at(Xf) * Wf
        pen = np.einsum("iap,jap,p->ij", Vf, Vf, w2)
        cons = np.einsum("iap,jap,p->ij", Sn, Vf, w2)          # ((grad^s phi_i) n) . phi_j
        A += cpen / hf * pen - cons - cons.T
    # pressure basis at the volume points (all functions kept)
    pv = []
    for e in range(d):
        s = S.pres[e]
        B, _ = splines.basis(s.knots, s.degree, X[:, e])
        pv.append(B[:, s.keep])
    shape = [pv[e].shape[1] for e in range(d)]
    multi = np.array(np.unravel_index(np.arange(int(np.prod(shape))), shape[::-1])).T[:, ::-1]
    Q = np.array([np.prod([pv[e][:, m[e]] for e in range(d)], axis=0) for m in multi])
    div = np.einsum("iaap->ip", G)
    Bm = -np.einsum("lp,jp,p->lj", Q, div, W)
    return A, Bm
