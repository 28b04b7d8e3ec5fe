"""Preconditioned MINRES (Paige & Saunders; the paper couples P_D with it in
Sec. 4 and runs it with tolerance 1e-8 from x0 = 0, Sec. 7).
Oracle: test infrastructure only.

Lanczos in the P-inner product with the tridiagonal QR by Givens rotations;
|eta| is the P^{-1}-norm of the current residual. Reading of the stopping
rule (the paper gives only the tolerance 1e-8): the recurrence estimate
|eta_j| / |eta_0| is compared with a threshold tau (initially tol); when it
falls below, the true residual ||b - A x_j||_2 / ||b||_2 is computed in FP64
and the solve ends if it is <= tol; otherwise tau <- 0.5 tau tol / true and
the iteration continues with its recurrences intact (true_check=True).
With true_check=False the estimate alone decides.

Pins (tests/test_oracle_minres.py): solution vs. numpy.linalg.solve on
random symmetric indefinite systems; |eta_j| equals the directly computed
||b - A x_j||_{P^{-1}} and never increases; with the ideal block
preconditioner diag(A, B A^{-1} B^T) a nonsingular saddle-point system is
solved in 3 iterations (three distinct eigenvalues, Murphy-Golub-Wathen).
"""
import math

import numpy as np


def minres(A, b, Pinv, tol=1e-8, maxit=1000, x0=None, history=None, true_check=False):
    """Returns (x, info) with info = dict(iters, status, eta_rel).
    A, Pinv: callables on 1-D float64 arrays. status: "converged", "maxit",
    "breakdown" (P not positive definite on the Krylov vector)."""
    b = np.asarray(b, float)
    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    v = b - A(x)                       # v_1 (unnormalized Lanczos vector, residual space)
    z = Pinv(v)                        # z_1 = P^{-1} v_1
    g2 = float(v @ z)
    if g2 < 0:
        return x, dict(iters=0, status="breakdown", eta_rel=float("nan"))
    gamma = math.sqrt(g2)              # gamma_1 = ||r_0||_{P^{-1}}
    if gamma == 0.0:
        return x, dict(iters=0, status="converged", eta_rel=0.0)
    eta0 = eta = gamma
    tau = tol
    bnorm = float(np.linalg.norm(b))
    v_old = np.zeros_like(b)
    w_old = np.zeros_like(b)
    w = np.zeros_like(b)
    gamma_old = 1.0
    c_old, c = 1.0, 1.0
    s_old, s = 0.0, 0.0
    if history is not None:
        history.append(1.0)
    for j in range(1, maxit + 1):
        z = z / gamma                               # normalized Lanczos vector
        Az = A(z)
        delta = float(Az @ z)
        v_new = Az - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = Pinv(v_new)
        g2 = float(v_new @ z_new)
        if g2 < 0:
            return x, dict(iters=j, status="breakdown", eta_rel=abs(eta) / eta0)
        gamma_new = math.sqrt(g2)
        # Givens: previous rotations applied to the new column of the tridiagonal matrix
        a0 = c * delta - c_old * s * gamma
        a1 = math.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new, s_new = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + c_new * eta * w_new
        eta = -s_new * eta
        if history is not None:
            history.append(abs(eta) / eta0)
        # shift
        v_old, v, z = v, v_new, z_new
        w_old, w = w, w_new
        gamma_old, gamma = gamma, gamma_new
        c_old, c = c, c_new
        s_old, s = s, s_new
        if abs(eta) / eta0 <= tau or gamma_new == 0.0:
            if not true_check or gamma_new == 0.0:
                return x, dict(iters=j, status="converged", eta_rel=abs(eta) / eta0)
            true = float(np.linalg.norm(b - A(x))) / (bnorm if bnorm > 0 else 1.0)
            if true <= tol:
                return x, dict(iters=j, status="converged", eta_rel=abs(eta) / eta0, true_rel=true)
            tau = 0.5 * tau * tol / true
    return x, dict(iters=maxit, status="maxit", eta_rel=abs(eta) / eta0)
