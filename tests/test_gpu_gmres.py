"""P_T / P_C block preconditioners and GMRES (paper Sec. 4, eq. P_T, eq. P_C and
the product form of P_C^{-1}) against the oracle: the applies element by
element (FP64, 1e-12), GMRES (left and flexible forms) iterations within one
of the oracle's (modified Gram-Schmidt there, classical Gram-Schmidt twice
here) with the FP64 true residual at the tolerance, and the mixed-precision
solve (split-TF32 FD, double-float matvec, flexible form) within two
iterations of the FP64 one."""
import numpy as np
import pytest

import synth
from oracle import gmres, stokes

from _helpers import gpu_problem, oracle_problem, problem_spec, max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

APPLY_CASES = [problem_spec(2, 2, 8), problem_spec(3, 2, 4), problem_spec(3, 3, (3, 4, 5)),
               problem_spec(2, 3, 6, "RT"), problem_spec(3, 2, 3, "RT")]


def _ids(c):
    return f"{c['disc']}-d{c['dim']}-p{c['p']}-{'x'.join(map(str, c['n_el']))}"


@pytest.mark.parametrize("spec", APPLY_CASES, ids=_ids)
@pytest.mark.parametrize("which", ["PT", "PC"])
def test_block_prec_apply_matches_oracle(spec, which):
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(spec, max_rhs=2)
    S = oracle_problem(spec)
    R = np.stack([synth.random_vector(900 + j, P.n_total) for j in range(2)])
    r = torch.tensor(R.reshape(-1), device="cuda")
    s = torch.empty_like(r)
    P.apply_block_prec(r, s, prec=fd.PREC_PT if which == "PT" else fd.PREC_PC)
    out = s.cpu().numpy().reshape(2, -1)
    ref_fn = stokes.apply_PT_inv if which == "PT" else stokes.apply_PC_inv
    for j in range(2):
        ref = ref_fn(S, R[j])
        for o0, o1 in zip(P.block_offsets[:-1], P.block_offsets[1:]):
            assert max_rel(out[j, o0:o1], ref[o0:o1]) <= 1e-12


@pytest.mark.parametrize("spec", [problem_spec(2, 2, 12), problem_spec(3, 2, 4), problem_spec(2, 2, 6, "RT")],
                         ids=_ids)
@pytest.mark.parametrize("which", ["PT", "PC"])
@pytest.mark.parametrize("flexible", [False, True], ids=["left", "flexible"])
def test_gmres_matches_oracle(spec, which, flexible):
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(spec, max_rhs=2)
    S = oracle_problem(spec)
    B = np.stack([synth.rhs(40 + j, P.block_sizes) for j in range(2)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.zeros_like(b)
    prec = fd.PREC_PT if which == "PT" else fd.PREC_PC
    info = P.solve_gmres(b, x, prec=prec, form=fd.GMRES_FLEXIBLE if flexible else fd.GMRES_LEFT, tol=1e-8,
                         maxit=300)
    X = x.cpu().numpy().reshape(2, -1)
    apply = stokes.apply_PT_inv if which == "PT" else stokes.apply_PC_inv
    for j in range(2):
        xo, io = gmres.gmres(lambda v: stokes.matvec(S, v), B[j], lambda v: apply(S, v), tol=1e-8, maxit=300,
                             true_check=True, flexible=flexible)
        assert info[j]["status"] == "OK"
        assert abs(info[j]["iterations"] - io["iters"]) <= 1
        assert info[j]["true_rel_res"] <= 1e-8
        res = np.linalg.norm(B[j] - stokes.matvec(S, X[j])) / np.linalg.norm(B[j])
        assert res <= 1e-8 and abs(res - info[j]["true_rel_res"]) <= 1e-10
        # the same velocity as the oracle's to the accuracy the tolerance allows (the
        # pressure is defined up to a constant)
        nv = P.block_offsets[-2]
        assert max_rel(X[j, :nv], xo[:nv]) <= 1e-5


def test_gmres_mixed_precision_and_restart():
    import paper_1712_00403_gb300 as fd
    spec = problem_spec(3, 2, 6)
    B = synth.rhs(77, gpu_problem(spec).block_sizes)
    its = {}
    mixed = dict(fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64)
    for name, kw, restart, form in (("f64", {}, 60, fd.GMRES_FLEXIBLE), ("mixed", mixed, 60, fd.GMRES_AUTO),
                                    ("f64-left", {}, 60, fd.GMRES_LEFT), ("restarted", {}, 8, fd.GMRES_LEFT)):
        P = gpu_problem(spec, **kw)
        b = torch.tensor(B, device="cuda")
        x = torch.zeros_like(b)
        info = P.solve_gmres(b, x, prec=fd.PREC_PT, form=form, tol=1e-8, maxit=400, restart=restart)[0]
        assert info["status"] == "OK" and info["true_rel_res"] <= 1e-8, (name, info)
        its[name] = info["iterations"]
    # split-TF32 FD apply in the flexible form: within two iterations of the FP64 flexible solve
    assert its["mixed"] <= its["f64"] + 2
    assert its["restarted"] >= its["f64-left"]


def test_gmres_zero_rhs_and_lockstep():
    import paper_1712_00403_gb300 as fd
    spec = problem_spec(2, 2, 10)
    P = gpu_problem(spec, max_rhs=3)
    B = np.stack([synth.rhs(5, P.block_sizes), np.zeros(P.n_total), synth.rhs(6, P.block_sizes)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.ones_like(b)
    info = P.solve_gmres(b, x, prec=fd.PREC_PC, tol=1e-8, maxit=200)
    X = x.cpu().numpy().reshape(3, -1)
    assert info[1]["status"] == "OK" and info[1]["iterations"] == 0 and np.all(X[1] == 0)
    for j in (0, 2):
        assert info[j]["status"] == "OK" and info[j]["true_rel_res"] <= 1e-8
        one = gpu_problem(spec)
        xj = torch.ones(P.n_total, dtype=torch.float64, device="cuda")
        i1 = one.solve_gmres(torch.tensor(B[j], device="cuda"), xj, prec=fd.PREC_PC, tol=1e-8, maxit=200)[0]
        assert abs(i1["iterations"] - info[j]["iterations"]) <= 1


def test_zero_initial_guess_spares_the_first_matvec():
    """x0 = 0 (the paper's start, Sec. 7) is detected on the device and the first
    residual taken as b. An x0 with one entry of 1e-300 leaves r0 = b to the last
    bit (its product with the operator vanishes against b's ulp, and underflows in
    the double-float split), so both starts take the same iterations; only the
    nonzero one pays for the first matvec's launches."""
    import paper_1712_00403_gb300 as fd
    spec = problem_spec(2, 2, 8)
    P = gpu_problem(spec)
    b = torch.tensor(synth.rhs(41, P.block_sizes), device="cuda")

    def run(solve, tiny):
        x = torch.zeros_like(b)
        if tiny:
            x[0] = 1e-300
        torch.cuda.synchronize()
        k0 = fd.kernel_launches()
        info = solve(b, x)[0]
        torch.cuda.synchronize()
        return info, fd.kernel_launches() - k0

    for solve in (lambda b, x: P.solve(b, x, tol=1e-8, maxit=300),
                  lambda b, x: P.solve_gmres(b, x, prec=fd.PREC_PT, tol=1e-8, maxit=300)):
        (iz, lz), (it, lt) = run(solve, False), run(solve, True)
        assert iz["status"] == "OK" and it["status"] == "OK"
        assert iz["iterations"] == it["iterations"]
        assert lt > lz, (lz, lt)
