"""Every status the C ABI declares, made to happen from the host without a
GPU fault: a non-finite right-hand side (NAN_DETECTED), a preconditioner that
is not positive definite on the right-hand side (BREAKDOWN), maxit
(MAXIT), an unreachable tolerance (STAGNATION), an allocation failure
injected on the host (OUT_OF_MEMORY, CUDA_ERROR, in fdst_setup and inside the
request server), a problem larger than the server's whole HBM budget
(ADMISSION_REJECTED), server cancellation of a queued and of an active
request (CANCELLED), the bounded-wait self-test (TIMEOUT), P_D^G on the
identity map (NOT_SUPPORTED). After each, the device keeps solving.
NOT_SPD (a univariate mass matrix that fails Cholesky) is exercised on the
host by tests/test_host_setup.py; INVALID_ARGUMENT by tests/test_abi.py."""
import numpy as np
import pytest

import synth
from oracle import stokes

from _helpers import gpu_problem, knots_of, oracle_problem, problem_spec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _still_solves():
    P = gpu_problem(problem_spec(2, 2, 6), max_rhs=1)
    b = torch.tensor(synth.rhs(5, P.block_sizes), device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8, maxit=300)[0]
    assert info["status"] == "OK" and info["true_rel_res"] <= 1e-8


def test_nan_right_hand_side_is_detected():
    P = gpu_problem(problem_spec(2, 2, 6), max_rhs=2)
    B = np.stack([synth.rhs(11 + j, P.block_sizes) for j in range(2)])
    B[1, 7] = np.nan
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.zeros_like(b)
    infos = P.solve(b, x, tol=1e-8, maxit=300)
    assert infos[0]["status"] == "OK" and infos[0]["true_rel_res"] <= 1e-8
    assert infos[1]["status"] == "NAN_DETECTED"
    _still_solves()


def test_indefinite_preconditioner_breaks_down():
    """RT with a penalty C_pen = 0.01, far below 5(alpha+1): the Nitsche factor K~
    is indefinite, so P_V has a negative eigenvalue. With b = P_D v for v the
    eigenvector of the most negative one, <P_D^{-1} b, b> = v^T P_D v < 0."""
    spec = problem_spec(2, 2, 4, "RT")
    S = stokes.build(knots_of(spec), 2, "RT", cpen=0.01)
    Pv = stokes.pv_matrix(S, 0)
    lam, V = np.linalg.eigh(Pv)
    assert lam[0] < 0
    b_h = np.zeros(S.n_total)
    b_h[:S.block_sizes[0]] = Pv @ V[:, 0]
    P = gpu_problem(spec, max_rhs=1, cpen=0.01)
    b = torch.tensor(b_h, device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8, maxit=50)[0]
    assert info["status"] == "BREAKDOWN"
    _still_solves()


def test_maxit_and_stagnation():
    P = gpu_problem(problem_spec(2, 2, 6), max_rhs=1)
    b = torch.tensor(synth.rhs(13, P.block_sizes), device="cuda")
    x = torch.zeros_like(b)
    assert P.solve(b, x, tol=1e-8, maxit=3)[0]["status"] == "MAXIT"
    # a tolerance below what FP64 reaches: the estimate meets its threshold, the
    # true residual never does, and after the restarts the solve reports stagnation
    x.zero_()
    info = P.solve(b, x, tol=1e-22, maxit=20000)[0]
    assert info["status"] == "STAGNATION", info
    assert info["true_rel_res"] <= 1e-12
    _still_solves()


@pytest.mark.parametrize("status", ["OUT_OF_MEMORY", "CUDA_ERROR"])
@pytest.mark.parametrize("nth", [1, 5])
def test_injected_allocation_failure_in_setup(status, nth):
    import paper_1712_00403_gb300 as fd
    code = {"OUT_OF_MEMORY": 3, "CUDA_ERROR": 4}[status]
    fd.inject_alloc_failure(nth, code)
    try:
        with pytest.raises(fd.FdstError) as e:
            gpu_problem(problem_spec(3, 2, 3), max_rhs=1)
        assert e.value.code == code
    finally:
        fd.inject_alloc_failure(0)
    _still_solves()


def _reqs(specs, seed0):
    out = []
    for k, spec in enumerate(specs):
        sizes = oracle_problem(spec).block_sizes
        out.append((spec, synth.rhs(seed0 + k, sizes)))
    return out


def _drain(server, n, limit=4000):
    for step in range(limit):
        _, _, fin = server.step(float(step))
        if fin >= n:
            return
    raise AssertionError("server did not finish")


def test_server_allocation_failure_and_admission_rejection():
    import paper_1712_00403_gb300 as fd
    spec = problem_spec(2, 2, (12, 9))
    reqs = _reqs([spec, spec], 800)
    # one request's handle set-up fails (the server's first device allocation); the next one is served
    server = fd.Server(max_active=2, iters_per_step=4, tol=1e-8, maxit=800)
    fd.inject_alloc_failure(1, 3)
    try:
        ids = [server.submit(knots_of(s), s["p"], b, 0.0) for s, b in reqs[:1]]
        _drain(server, 1)
    finally:
        fd.inject_alloc_failure(0)
    ids += [server.submit(knots_of(s), s["p"], b, 1.0) for s, b in reqs[1:]]
    _drain(server, 2)
    assert server.result(ids[0])["status"] == "OUT_OF_MEMORY"
    r = server.result(ids[1])
    assert r["status"] == "OK" and r["true_rel_res"] <= 1e-8
    held = server.stats()["bytes_held"]          # the one idle handle
    server.close()
    assert held > 0
    # a budget below one handle's size: the request can never be admitted
    server = fd.Server(max_active=2, hbm_budget_bytes=held // 2, iters_per_step=4, tol=1e-8, maxit=800)
    rid = server.submit(knots_of(spec), spec["p"], reqs[0][1], 0.0)
    _drain(server, 1)
    assert server.result(rid)["status"] == "ADMISSION_REJECTED"
    assert server.stats()["bytes_held"] == 0
    server.close()
    _still_solves()


def test_server_cancel_queued_and_active():
    import paper_1712_00403_gb300 as fd
    specs = [problem_spec(2, 2, (12, 9)), problem_spec(2, 3, (8, 8)), problem_spec(2, 2, (10, 7))]
    reqs = _reqs(specs, 820)
    server = fd.Server(max_active=1, iters_per_step=2, tol=1e-8, maxit=800)
    ids = [server.submit(knots_of(s), s["p"], b, 0.0) for s, b in reqs]
    a, q, _ = server.step(0.0)
    assert a == 1 and q == 2
    server.cancel(ids[0])          # active: retired at the next step
    server.cancel(ids[1])          # queued: finished at once
    r1 = server.result(ids[1])
    assert r1 is not None and r1["status"] == "CANCELLED"
    assert server.result(ids[0]) is None
    _drain(server, 3)
    assert server.result(ids[0])["status"] == "CANCELLED"
    r2 = server.result(ids[2])
    assert r2["status"] == "OK" and r2["true_rel_res"] <= 1e-8
    server.cancel(ids[2])          # finished: left as it is
    assert server.result(ids[2])["status"] == "OK"
    with pytest.raises(fd.FdstError):
        server.cancel(12345)
    server.close()


def test_bounded_wait_reports_timeout():
    import paper_1712_00403_gb300 as fd
    status, gave_up, seconds = fd.check_bounded_wait()
    assert status == "TIMEOUT" and gave_up
    _still_solves()


def test_geometry_variant_on_identity_map_is_not_supported():
    import paper_1712_00403_gb300 as fd
    with pytest.raises(fd.FdstError) as e:
        gpu_problem(problem_spec(3, 2, 3), variant=fd.VARIANT_PD_GEO)
    assert fd.STATUS[e.value.code] == "NOT_SUPPORTED"
