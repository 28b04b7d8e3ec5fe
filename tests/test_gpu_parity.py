"""CUDA path vs. the CPU FP64 oracle, through the C ABI.

Bar (FP64 path): element-wise relative difference max|y - y_ref| / max|y_ref|
of every block <= 1e-12 (an FD apply with n_v > 256: u kappa(Delta), see
fd64_bar) for the FD
preconditioner apply (Algorithm 1) and for the Kronecker Stokes matvec
(Sec. 3); MINRES (Sec. 4, Sec. 7) reaches the same iteration count within
one iteration and a true relative residual <= 1e-8.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import minres, stokes

from _helpers import gpu_problem, oracle_problem, problem_spec, max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    problem_spec(2, 2, 16),            # 2D unit square, p=2, 16x16 (n_v = 32, n_q = 18)
    problem_spec(2, 3, (5, 9)),        # 2D, unequal directions
    problem_spec(3, 2, 4),             # 3D small cube
    problem_spec(3, 3, (3, 4, 6)),     # 3D, three different sizes (index-order check)
    problem_spec(3, 2, 9),             # 3D, rows span several tiles with a ragged tail
    problem_spec(2, 2, 6, "RT"),       # 2D Raviart-Thomas with Nitsche terms
    problem_spec(2, 4, (4, 7), "RT"),
    problem_spec(3, 2, 4, "RT"),       # 3D Raviart-Thomas: Nitsche terms in two directions per component
    problem_spec(3, 3, (3, 4, 5), "RT"),
    problem_spec(2, 3, (26, 5)),       # n_v = 53 > 48: Householder + implicit-QL eigensolver path
    problem_spec(2, 2, 140),           # n_v = 280: FP64 contraction with K and N above 256
    problem_spec(3, 6, (90, 17, 23)),  # a batched-workload-sized instance: p = 6, n_v = 184 x 38 x 50
    problem_spec(2, 1, (1, 3)),        # degenerate: one element, p = 1 (one velocity function across it)
    problem_spec(3, 1, (1, 2, 3)),
    problem_spec(3, 2, (1, 1, 5)),     # two directions of a single element
    problem_spec(2, 1, 1, "RT"),       # the smallest Raviart-Thomas system (8 unknowns)
    problem_spec(3, 1, (1, 2, 2), "RT"),
]


def _ids(c):
    return f"{c['disc']}-d{c['dim']}-p{c['p']}-{'x'.join(map(str, c['n_el']))}"


def fd64_bar(S):
    """Bar of an FP64 FD apply: 1e-12, or u kappa(Delta) where that is larger.
    The apply solves P s = r through the pencils' eigendecompositions; two
    backward-stable eigensolvers give results that differ by up to about
    u kappa (u = 2^-53, kappa = largest over smallest entry of Delta = sum_d
    c_d lam_d): the oracle's own LAPACK and Cholesky + symmetric-QR routes
    differ by 2.4e-12 at n_v = 280 (u kappa = 1.8e-11) and by 1.6e-13 at
    n_v = 128 (u kappa = 3.8e-12)."""
    u = 2.0 ** -53
    kappa = 0.0
    for k in range(S.dim):
        Ks, Ms, coef = stokes.pv_pencils(S, k)
        lam = [scipy.linalg.eigh(K, M, eigvals_only=True) for K, M in zip(Ks, Ms)]
        kappa = max(kappa, sum(c * l.max() for c, l in zip(coef, lam)) / sum(c * l.min() for c, l in zip(coef, lam)))
    return max(1e-12, u * kappa)


@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_fd_apply_f64_matches_oracle(spec):
    P = gpu_problem(spec, max_rhs=3)
    S = oracle_problem(spec)
    bar = fd64_bar(S) if max(S.vel_shapes[0]) > 256 else 1e-12
    assert P.block_sizes == S.block_sizes
    R = np.stack([synth.random_vector(100 + j, P.n_total) for j in range(3)])
    r = torch.tensor(R.reshape(-1), device="cuda")
    s = torch.empty_like(r)
    P.apply_prec(r, s)
    out = s.cpu().numpy().reshape(3, -1)
    for j in range(3):
        ref = stokes.apply_PD_inv(S, R[j], "fd")
        for b, (o0, o1) in enumerate(zip(P.block_offsets[:-1], P.block_offsets[1:])):
            assert max_rel(out[j, o0:o1], ref[o0:o1]) <= bar, (j, b)


@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_matvec_f64_matches_oracle(spec):
    P = gpu_problem(spec, max_rhs=2, viscosity=1.0)
    S = oracle_problem(spec)
    X = np.stack([synth.random_vector(300 + j, P.n_total) for j in range(2)])
    x = torch.tensor(X.reshape(-1), device="cuda")
    y = torch.empty_like(x)
    P.matvec(x, y)
    out = y.cpu().numpy().reshape(2, -1)
    for j in range(2):
        ref = stokes.matvec(S, X[j])
        for o0, o1 in zip(P.block_offsets[:-1], P.block_offsets[1:]):
            assert max_rel(out[j, o0:o1], ref[o0:o1]) <= 1e-12


def test_matvec_constant_pressure_kernel():
    spec = problem_spec(3, 2, 5)
    P = gpu_problem(spec)
    x = torch.zeros(P.n_total, dtype=torch.float64, device="cuda")
    x[P.block_offsets[-2]:] = 1.0
    y = torch.empty_like(x)
    P.matvec(x, y)
    assert float(y.abs().max()) < 1e-12


@pytest.mark.parametrize("spec", [problem_spec(2, 2, 16), problem_spec(3, 2, 4), problem_spec(2, 2, 8, "RT"),
                                  problem_spec(3, 2, 4, "RT")], ids=_ids)
def test_minres_f64_matches_oracle(spec):
    P = gpu_problem(spec, max_rhs=2)
    S = oracle_problem(spec)
    B = np.stack([synth.rhs(1 + j, P.block_sizes) for j in range(2)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8, maxit=500)
    X = x.cpu().numpy().reshape(2, -1)
    for j in range(2):
        xo, io = minres.minres(lambda v: stokes.matvec(S, v), B[j], lambda v: stokes.apply_PD_inv(S, v),
                               tol=1e-8, maxit=500, true_check=True)
        assert info[j]["status"] == "OK"
        assert abs(info[j]["iterations"] - io["iters"]) <= 1
        # the estimate-only stopping rule: the oracle's recurrence without the true-residual check
        _, ie = minres.minres(lambda v: stokes.matvec(S, v), B[j], lambda v: stokes.apply_PD_inv(S, v),
                              tol=1e-8, maxit=500, true_check=False)
        assert abs(info[j]["iterations_estimate"] - ie["iters"]) <= 1
        assert info[j]["iterations_estimate"] <= info[j]["iterations"]
        assert info[j]["true_rel_res"] <= 1e-8
        res = np.linalg.norm(B[j] - stokes.matvec(S, X[j])) / np.linalg.norm(B[j])
        assert res <= 1e-8
        assert abs(res - info[j]["true_rel_res"]) <= 1e-10


def test_multi_rhs_equals_single():
    spec = problem_spec(3, 2, 5)
    P4 = gpu_problem(spec, max_rhs=4)
    P1 = gpu_problem(spec, max_rhs=1)
    B = np.stack([synth.rhs(40 + j, P4.block_sizes) for j in range(4)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.zeros_like(b)
    info4 = P4.solve(b, x, tol=1e-8, maxit=300)
    X4 = x.cpu().numpy().reshape(4, -1)
    for j in range(4):
        bj = torch.tensor(B[j], device="cuda")
        xj = torch.zeros_like(bj)
        info1 = P1.solve(bj, xj, tol=1e-8, maxit=300)
        assert info1[0]["iterations"] == info4[j]["iterations"]
        assert max_rel(X4[j], xj.cpu().numpy()) <= 1e-13


def test_staggered_stops_and_resumes_equal_single_solves():
    """Right-hand sides whose recurrence estimates meet the threshold at different
    iterations sit stopped for different numbers of iterations (odd and even) while
    the others run, then resume after the true-residual check. MINRES exchanges the
    roles of (v, v_old) and (w, w_old) by pointer every iteration, so a stopped one
    has its slices exchanged back before it resumes: each must equal its own
    single-right-hand-side solve (split-TF32 FD, double-float matvec)."""
    import paper_1712_00403_gb300 as fd
    spec = problem_spec(3, 2, 16)
    kw = dict(fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64)
    P6 = gpu_problem(spec, max_rhs=6, **kw)
    P1 = gpu_problem(spec, max_rhs=1, **kw)
    B = np.stack([synth.rhs(900 + j, P6.block_sizes) * 10.0 ** (j - 2) for j in range(6)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.zeros_like(b)
    info6 = P6.solve(b, x, tol=1e-8, maxit=500)
    est = [i["iterations_estimate"] for i in info6]
    assert max(est) > min(est), est                                    # staggered stops
    assert all(i["iterations"] > i["iterations_estimate"] for i in info6), info6   # every one resumed
    X6 = x.cpu().numpy().reshape(6, -1)
    for j in range(6):
        bj = torch.tensor(B[j], device="cuda")
        xj = torch.zeros_like(bj)
        info1 = P1.solve(bj, xj, tol=1e-8, maxit=500)[0]
        assert info6[j]["status"] == "OK" and info6[j]["true_rel_res"] <= 1e-8
        assert info1["iterations"] == info6[j]["iterations"], (j, info1, info6[j])
        assert max_rel(X6[j], xj.cpu().numpy()) <= 1e-13


def test_host_entry_points_match_device():
    spec = problem_spec(2, 2, 8)
    P = gpu_problem(spec)
    bh = synth.rhs(5, P.block_sizes)
    xh = np.zeros_like(bh)
    info_h = P.solve_host(bh, xh, tol=1e-8, maxit=300)
    b = torch.tensor(bh, device="cuda")
    x = torch.zeros_like(b)
    info_d = P.solve(b, x, tol=1e-8, maxit=300)
    assert info_h[0]["iterations"] == info_d[0]["iterations"]
    assert max_rel(xh, x.cpu().numpy()) <= 1e-14
    # zero initial guess: whatever the output array holds is never read
    xz = np.full_like(bh, np.nan)
    info_z = P.solve_host(bh, xz, tol=1e-8, maxit=300, zero_guess=True)
    assert info_z[0]["iterations"] == info_d[0]["iterations"]
    assert np.array_equal(xz, xh)
    sh = np.empty_like(bh)
    P.apply_prec_host(bh, sh)
    s = torch.empty_like(b)
    P.apply_prec(b, s)
    assert max_rel(sh, s.cpu().numpy()) <= 1e-15


@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_matvec_df64_matches_oracle(spec):
    """Double-float matvec (FP32 pairs, error-free transformations) within the FP64 bar."""
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(spec, max_rhs=2, matvec_precision=fd.MV_DF64)
    S = oracle_problem(spec)
    X = np.stack([synth.random_vector(700 + j, P.n_total) for j in range(2)])
    x = torch.tensor(X.reshape(-1), device="cuda")
    y = torch.empty_like(x)
    P.matvec(x, y)
    out = y.cpu().numpy().reshape(2, -1)
    for j in range(2):
        ref = stokes.matvec(S, X[j])
        for o0, o1 in zip(P.block_offsets[:-1], P.block_offsets[1:]):
            assert max_rel(out[j, o0:o1], ref[o0:o1]) <= 1e-12


@pytest.mark.parametrize("spec", [problem_spec(3, 2, 6), problem_spec(2, 2, 16)], ids=_ids)
def test_minres_df64_matvec_matches_f64(spec):
    import paper_1712_00403_gb300 as fd
    Pd = gpu_problem(spec, max_rhs=2, matvec_precision=fd.MV_DF64)
    Pf = gpu_problem(spec, max_rhs=2, matvec_precision=fd.MV_F64)
    B = np.stack([synth.rhs(80 + j, Pd.block_sizes) for j in range(2)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    xd, xf = torch.zeros_like(b), torch.zeros_like(b)
    idd = Pd.solve(b, xd, tol=1e-8, maxit=500)
    iff = Pf.solve(b, xf, tol=1e-8, maxit=500)
    for a, c in zip(idd, iff):
        assert a["status"] == "OK" and a["true_rel_res"] <= 1e-8
        assert abs(a["iterations"] - c["iterations"]) <= 1


@pytest.mark.parametrize("spec", [problem_spec(3, 2, 5), problem_spec(2, 3, (5, 9))], ids=_ids)
def test_matvec_df64_six_rhs_matches_oracle(spec):
    """Six right-hand sides through the double-float matvec: every right-hand
    side within the FP64 bar, and a solve with six right-hand sides equals the
    six solves done one at a time."""
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(spec, max_rhs=6, matvec_precision=fd.MV_DF64)
    S = oracle_problem(spec)
    X = np.stack([synth.random_vector(720 + j, P.n_total) for j in range(6)])
    x = torch.tensor(X.reshape(-1), device="cuda")
    y = torch.empty_like(x)
    P.matvec(x, y)
    out = y.cpu().numpy().reshape(6, -1)
    for j in range(6):
        ref = stokes.matvec(S, X[j])
        for o0, o1 in zip(P.block_offsets[:-1], P.block_offsets[1:]):
            assert max_rel(out[j, o0:o1], ref[o0:o1]) <= 1e-12, j
    B = np.stack([synth.rhs(90 + j, P.block_sizes) for j in range(6)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    xs = torch.zeros_like(b)
    many = P.solve(b, xs, tol=1e-8, maxit=500)
    P1 = gpu_problem(spec, max_rhs=1, matvec_precision=fd.MV_DF64)
    for j in range(6):
        bj = torch.tensor(B[j], device="cuda")
        xj = torch.zeros_like(bj)
        one = P1.solve(bj, xj, tol=1e-8, maxit=500)[0]
        assert many[j]["status"] == "OK" and many[j]["true_rel_res"] <= 1e-8
        assert abs(many[j]["iterations"] - one["iterations"]) <= 1
        assert max_rel(xs.cpu().numpy().reshape(6, -1)[j], xj.cpu().numpy()) <= 1e-7
