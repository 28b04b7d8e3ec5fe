"""Batched solves (fdst_batch_*): uneven problems advanced together by grouped
launches under a CUDA graph give each problem the result it gets alone
(same iteration count within one, solution within 1e-7 relative, true
residual <= 1e-8), for the FP64 and the split-TF32 FD apply."""
import numpy as np
import pytest

import synth
from oracle import minres, stokes

from _helpers import gpu_problem, oracle_problem, problem_spec, max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPECS = [problem_spec(3, 2, (4, 5, 6)), problem_spec(3, 3, (3, 3, 7)), problem_spec(2, 2, (12, 9)),
         problem_spec(3, 2, (6, 4, 3)), problem_spec(2, 4, (5, 8))]


@pytest.mark.parametrize("tc", [False, True], ids=["f64", "tf32"])
def test_batch_equals_individual_solves(tc):
    import paper_1712_00403_gb300 as fd
    prec = fd.FD_TF32X3 if tc else fd.FD_F64
    probs = [gpu_problem(s, fd_precision=prec, matvec_precision=fd.MV_DF64) for s in SPECS]
    bs = [torch.tensor(synth.rhs(401 + i, p.block_sizes), device="cuda") for i, p in enumerate(probs)]
    batch = fd.Batch(probs, autotune=True)
    info = batch.info()
    assert info["band_threads"] in (128, 256)
    if tc:
        assert 2 <= info["tc_ring"] <= 4
    xs = [torch.zeros_like(b) for b in bs]
    res = batch.solve(bs, xs, tol=1e-8, maxit=500)
    res2 = batch.solve(bs, [torch.zeros_like(b) for b in bs], tol=1e-8, maxit=500)   # graph replay again
    batch.close()
    for i, p in enumerate(probs):
        x1 = torch.zeros_like(bs[i])
        single = p.solve(bs[i], x1, tol=1e-8, maxit=500)[0]
        assert res[i]["status"] == "OK" and res[i]["true_rel_res"] <= 1e-8
        assert abs(res[i]["iterations"] - single["iterations"]) <= 1
        assert res2[i]["iterations"] == res[i]["iterations"]
        assert max_rel(xs[i].cpu().numpy(), x1.cpu().numpy()) <= 1e-7
    assert fd.device_error() == 0


def test_batch_f64_matches_oracle():
    import paper_1712_00403_gb300 as fd
    spec = SPECS[0]
    probs = [gpu_problem(s, fd_precision=fd.FD_F64, matvec_precision=fd.MV_DF64) for s in SPECS[:3]]
    bs = [torch.tensor(synth.rhs(501 + i, p.block_sizes), device="cuda") for i, p in enumerate(probs)]
    xs = [torch.zeros_like(b) for b in bs]
    batch = fd.Batch(probs, autotune=False)
    res = batch.solve(bs, xs, tol=1e-8, maxit=500)
    batch.close()
    S = oracle_problem(spec)
    xo, io = minres.minres(lambda v: stokes.matvec(S, v), bs[0].cpu().numpy(), lambda v: stokes.apply_PD_inv(S, v),
                           tol=1e-8, maxit=500, true_check=True)
    assert abs(res[0]["iterations"] - io["iters"]) <= 1
    assert max_rel(xs[0].cpu().numpy(), xo) <= 1e-7


@pytest.mark.parametrize("mode", ["streamed", "resident_b", "resident_b_tmem_a"])
def test_batch_feeding_modes_give_the_same_solves(mode):
    """Every feeding mode the autotuner chooses among (B streamed with A, B
    resident in shared memory over the batch's problem table, A's TF32 pieces in
    tensor memory) forced on every contraction step: the batched split-TF32 solve
    equals each problem's solve alone, and the tuning reads back as set."""
    import paper_1712_00403_gb300 as fd
    probs = [gpu_problem(s, fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64) for s in SPECS]
    bs = [torch.tensor(synth.rhs(601 + i, p.block_sizes), device="cuda") for i, p in enumerate(probs)]
    batch = fd.Batch(probs, autotune=False)
    nsteps = len(batch.info()["step_modes"])
    rings = [2 if mode == "streamed" else 0] * nsteps
    batch.set_tuning([mode] * nsteps, rings)
    info = batch.info()
    assert info["step_modes"] == [mode] * nsteps and info["step_rings"] == rings
    xs = [torch.zeros_like(b) for b in bs]
    res = batch.solve(bs, xs, tol=1e-8, maxit=500)
    batch.close()
    for i, p in enumerate(probs):
        x1 = torch.zeros_like(bs[i])
        single = p.solve(bs[i], x1, tol=1e-8, maxit=500)[0]
        assert res[i]["status"] == "OK" and res[i]["true_rel_res"] <= 1e-8
        assert abs(res[i]["iterations"] - single["iterations"]) <= 1
        assert max_rel(xs[i].cpu().numpy(), x1.cpu().numpy()) <= 1e-7
    assert fd.device_error() == 0


def test_batch_set_tuning_rejects_what_does_not_fit():
    import paper_1712_00403_gb300 as fd
    probs = [gpu_problem(s, fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64) for s in SPECS[:2]]
    batch = fd.Batch(probs, autotune=False)
    n = len(batch.info()["step_modes"])
    with pytest.raises(ValueError):
        batch.set_tuning(["streamed"] * (n - 1), [0] * n)
    with pytest.raises(fd.FdstError) as e:
        batch.set_tuning(["streamed"] * n, [-1] * n)
    assert fd.STATUS[e.value.code] == "INVALID_ARGUMENT"
    with pytest.raises(fd.FdstError) as e:
        batch.set_tuning(["streamed"] * n, [1] * n)   # one stage: below the two the pipeline needs
    assert fd.STATUS[e.value.code] == "NOT_SUPPORTED"
    batch.close()
    probs64 = [gpu_problem(s, fd_precision=fd.FD_F64) for s in SPECS[:2]]
    b64 = fd.Batch(probs64, autotune=False)
    with pytest.raises(fd.FdstError) as e:
        b64.set_tuning(["streamed"] * len(b64.info()["step_modes"]), [0] * len(b64.info()["step_modes"]))
    assert fd.STATUS[e.value.code] == "NOT_SUPPORTED"
    b64.close()
