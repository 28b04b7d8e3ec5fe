"""Kronecker-product identities and the Fast Diagonalization solve.
Oracle: test infrastructure only.

Layout (Sec. 2.3, vec operator): a tensor X in R^{n1 x n2 (x n3)} is stored as
vec(X) with i1 fastest; in numpy it is the C-ordered array of shape
(n3, n2, n1) (or (n2, n1) in 2D). ``factors`` are always listed in mode order
[A1, A2, A3]; the matrix they stand for is A3 (x) A2 (x) A1 (eq. kronvec).

Pins (tests/test_oracle_kron.py): mode products vs. the explicit np.kron
matrix; the FD solve vs. a dense LU solve of the assembled Kronecker sum
(eq. sylv_eq) on tiny grids; U^T M U = I and U^T K U = Lambda (eq. eig_dec);
the banded P_Q solve vs. dense inverse.
"""
import numpy as np
import scipy.linalg as sla


def mode_product(X, A, mode):
    """[X x_mode A]: contract index i_mode of X (mode 1 = fastest axis) with A's columns."""
    axis = X.ndim - mode          # mode 1 -> last numpy axis
    Y = np.tensordot(A, X, axes=([1], [axis]))   # new axis first
    return np.moveaxis(Y, 0, axis)


def kron_apply(factors, x):
    """(A_d (x) ... (x) A_1) x via mode products (eq. kronvec)."""
    shape = tuple(A.shape[1] for A in reversed(factors))
    X = np.asarray(x, float).reshape(shape)
    for mode, A in enumerate(factors, start=1):
        X = mode_product(X, A, mode)
    return X.reshape(-1)


def kron_matrix(factors):
    """Explicit A_d (x) ... (x) A_1 (tiny sizes only)."""
    out = np.ones((1, 1))
    for A in reversed(factors):
        out = np.kron(out, A)
    return out


def kron_sum_terms(Ks, Ms, coef):
    """Terms of sum_d coef[d] * (x)_{e} (K_e if e == d else M_e), mode order."""
    dim = len(Ks)
    return [(coef[d], [Ks[e] if e == d else Ms[e] for e in range(dim)]) for d in range(dim)]


def kron_sum_matrix(Ks, Ms, coef):
    """Assembled Kronecker sum R of eq. sylv_eq, with per-direction coefficients."""
    return sum(c * kron_matrix(f) for c, f in kron_sum_terms(Ks, Ms, coef))


def kron_sum_apply(Ks, Ms, coef, x):
    return sum(c * kron_apply(f, x) for c, f in kron_sum_terms(Ks, Ms, coef))


def gen_eig(K, M):
    """Generalized symmetric eigenproblem K U = M U diag(lam), U^T M U = I (eq. eig_dec).
    LAPACK (scipy.linalg.eigh) serves as the library step, as Matlab eig did in the paper."""
    lam, U = sla.eigh(K, M)
    return lam, U


def fd_solve(Ks, Ms, coef, t, eig=None):
    """Algorithm 1 (FD): q = (U_d..U_1) Delta^{-1} (U_d..U_1)^T t with
    Delta = sum_d coef[d] lam_d (on index i_d). Reading: the Kronecker order
    U3 (x) U2 (x) U1 of the factorization is used (the algorithm lists the
    factors in the opposite order, which is inconsistent with eq. sylv_eq)."""
    if eig is None:
        eig = [gen_eig(K, M) for K, M in zip(Ks, Ms)]
    Us = [U for _, U in eig]
    lams = [lam for lam, _ in eig]
    tt = kron_apply([U.T for U in Us], t)
    shape = tuple(len(l) for l in reversed(lams))
    D = np.zeros(shape)
    for d, lam in enumerate(lams):
        bshape = [1] * len(lams)
        bshape[len(lams) - 1 - d] = len(lam)
        D = D + coef[d] * lam.reshape(bshape)
    qt = tt.reshape(shape) / D
    return kron_apply(Us, qt.reshape(-1))


def dense_solve(Ks, Ms, coef, t):
    """Direct dense LU solve of R q = t (the definition the FD method reaches exactly)."""
    R = kron_sum_matrix(Ks, Ms, coef)
    return sla.lu_solve(sla.lu_factor(R), t)


def banded_of(A):
    """Upper band storage of a symmetric banded matrix for solveh_banded."""
    n = A.shape[0]
    nz = np.nonzero(np.abs(A) > 0)
    bw = int(np.max(np.abs(nz[0] - nz[1]))) if len(nz[0]) else 0
    ab = np.zeros((bw + 1, n))
    for k in range(bw + 1):
        ab[bw - k, k:] = np.diagonal(A, k)
    return ab


def kron_mass_solve(Ms, t):
    """(M_d (x) ... (x) M_1)^{-1} t by banded Cholesky solves mode by mode
    (eq. kron_vec_sol; the direct O(p n_Q) route of Sec. 5.2)."""
    shape = tuple(M.shape[0] for M in reversed(Ms))
    X = np.asarray(t, float).reshape(shape)
    for mode, M in enumerate(Ms, start=1):
        axis = X.ndim - mode
        Xm = np.moveaxis(X, axis, 0)
        sol = sla.solveh_banded(banded_of(M), Xm.reshape(M.shape[0], -1), lower=False)
        X = np.moveaxis(sol.reshape(Xm.shape), 0, axis)
    return X.reshape(-1)
