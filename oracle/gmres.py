"""Left-preconditioned GMRES (Saad & Schultz; the paper couples the block
triangular P_T and the constraint P_C with it, Sec. 4, tolerance 1e-8 from
x0 = 0, Sec. 7). Oracle: test infrastructure only.

Arnoldi on P^{-1} A with modified Gram-Schmidt, the Hessenberg least-squares
problem reduced by Givens rotations, so that |g_{j+1}| is the 2-norm of the
preconditioned residual P^{-1}(b - A x_j). Reading of the stopping rule (the
paper gives the tolerance only; the same reading as for MINRES): the estimate
|g_{j+1}| / ||P^{-1} b|| is compared with a threshold tau (initially tol);
when it falls below, x_j is formed and the true residual ||b - A x_j||_2 /
||b||_2 is computed in FP64; the solve ends if it is <= tol, otherwise
tau <- 0.5 tau tol / true and the Arnoldi process continues with its basis
intact (true_check=True). With true_check=False the estimate alone decides.
The basis holds at most `restart` vectors; when it is full, x is formed and
the process starts again from the new residual.

flexible=True gives the right-preconditioned flexible form (Saad's FGMRES):
Arnoldi on A with z_j = P^{-1} v_j kept, x_j = x_0 + Z_j y_j, so that the
estimate |g_{j+1}| / ||b|| is the unpreconditioned relative residual and the
Arnoldi relation A Z_j = V_{j+1} H_j holds however P^{-1} was evaluated (the
form for preconditioners applied in reduced precision).

Pins (tests/test_oracle_gmres.py): solution vs. numpy.linalg.solve on random
nonsymmetric systems (exact after n steps); the estimate equals the directly
computed ||P^{-1}(b - A x_j)|| and never increases; with the ideal block
triangular preconditioner (P_V = A, P_Q = B A^{-1} B^T) P^{-1} A has minimal
polynomial (z - 1)^2 and GMRES stops after 2 steps; with the ideal constraint
preconditioner P_C equals A and GMRES stops after 1 step.
"""
import numpy as np


def gmres(A, b, Pinv, tol=1e-8, maxit=1000, restart=200, x0=None, history=None, true_check=False, flexible=False):
    """Returns (x, info) with info = dict(iters, status, est_rel, true_rel).
    A, Pinv: callables on 1-D float64 arrays. status: "converged" or "maxit"."""
    b = np.asarray(b, float)
    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    nb = np.linalg.norm(b)
    beta_ref = nb if flexible else np.linalg.norm(Pinv(b))
    if nb == 0.0 or beta_ref == 0.0:
        return np.zeros_like(b), dict(iters=0, status="converged", est_rel=0.0, true_rel=0.0)
    tau = tol
    it = 0
    est = np.inf
    while it < maxit:
        r = (b - A(x)) if flexible else Pinv(b - A(x))
        beta = np.linalg.norm(r)
        m = min(restart, maxit - it)
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size)) if flexible else None
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        if beta == 0.0:
            return x, dict(iters=it, status="converged", est_rel=0.0, true_rel=np.linalg.norm(b - A(x)) / nb)
        V[0] = r / beta
        j = 0
        done = False
        while j < m:
            if flexible:
                Z[j] = Pinv(V[j])
                w = A(Z[j])
            else:
                w = Pinv(A(V[j]))
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # earlier rotations on the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j, j] / den, H[j + 1, j] / den)
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            it += 1
            est = abs(g[j]) / beta_ref
            if history is not None:
                history.append(est)
            if est <= tau:
                xj = x + _combine(Z if flexible else V, H, g, j)
                if not true_check:
                    x = xj
                    done = True
                    break
                true = np.linalg.norm(b - A(xj)) / nb
                if true <= tol:
                    x = xj
                    done = True
                    break
                tau = 0.5 * tau * tol / true
            if it >= maxit:
                break
        if done:
            return x, dict(iters=it, status="converged", est_rel=est,
                           true_rel=np.linalg.norm(b - A(x)) / nb)
        x = x + _combine(Z if flexible else V, H, g, j)
    return x, dict(iters=it, status="maxit", est_rel=est, true_rel=np.linalg.norm(b - A(x)) / nb)


def _combine(V, H, g, j):
    """V_j y (or Z_j y) with y the solution of the rotated (upper triangular) j x j system."""
    y = np.zeros(j)
    for i in range(j - 1, -1, -1):
        y[i] = (g[i] - np.dot(H[i, i + 1:j], y[i + 1:j])) / H[i, i]
    return y @ V[:j]
