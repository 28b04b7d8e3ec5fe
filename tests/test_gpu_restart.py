"""MINRES restart from the current iterate when the recurrence drifts from the
true residual (reading of the stopping rule, Sec. 4/7): a high-degree
anisotropic instance (p=6, 90x16x52 elements) whose double-float recurrence
reaches a 1e-16 estimate while its FP64 true residual stays above 1e-8 must
still reach the tolerance, alone, in a batch and through the request server,
within a few iterations of the FP64-matvec solve."""
import numpy as np
import pytest

import synth

from _helpers import knots_of, problem_spec, max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPEC = problem_spec(3, 6, (90, 16, 52))


def _solve(fd, mv, prec=None):
    prec = fd.FD_TF32X3 if prec is None else prec
    P = fd.Stokes(knots_of(SPEC), SPEC["p"], fd_precision=prec, matvec_precision=mv)
    b = torch.tensor(synth.rhs(426, P.block_sizes), device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8, maxit=400)[0]
    return P, b, x, info


def test_restart_reaches_tolerance_alone():
    import paper_1712_00403_gb300 as fd
    P64, b, x64, i64 = _solve(fd, fd.MV_F64)
    for prec in (fd.FD_F64, fd.FD_TF32X3):
        P, b, x, info = _solve(fd, fd.MV_DF64, prec)
        assert info["status"] == "OK" and info["true_rel_res"] <= 1e-8
        assert info["iterations"] <= i64["iterations"] + 10
        # FP64 residual of the returned iterate through the FP64-matvec handle
        y = torch.empty_like(b)
        P64.matvec(x, y)
        assert float(torch.linalg.norm(b - y) / torch.linalg.norm(b)) <= 1e-8 * 1.01
        assert max_rel(x.cpu().numpy(), x64.cpu().numpy()) <= 1e-5
        P.close()
    P64.close()


def test_restart_in_batch_and_server():
    import paper_1712_00403_gb300 as fd
    small = problem_spec(3, 2, (4, 5, 3))
    probs = [fd.Stokes(knots_of(s), s["p"], fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64)
             for s in (SPEC, small)]
    bs = [torch.tensor(synth.rhs(426 + i, p.block_sizes), device="cuda") for i, p in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    batch = fd.Batch(probs, autotune=False)
    res = batch.solve(bs, xs, tol=1e-8, maxit=400)
    batch.close()
    for r in res:
        assert r["status"] == "OK" and r["true_rel_res"] <= 1e-8
    server = fd.Server(max_active=2, iters_per_step=4, tol=1e-8, maxit=400)
    rid = server.submit(knots_of(SPEC), SPEC["p"], bs[0].cpu().numpy(), 0.0)
    step = 0
    while True:
        _, _, finished = server.step(float(step))
        step += 1
        if finished == 1:
            break
        assert step < 1000
    r = server.result(rid)
    server.close()
    assert r["status"] == "OK" and r["true_rel_res"] <= 1e-8
    assert max_rel(r["x"], xs[0].cpu().numpy()) <= 1e-6
    for p in probs:
        p.close()
