"""Request server (fdst_server_*): requests that arrive while others are on
the GPU join between steps; every result equals the problem's solve alone
(iterations within one, solution within 1e-7 relative, true residual <= 1e-8,
and the true residual under the oracle's FP64 operator <= 1e-8 as well);
the active-slot limit and the HBM budget hold; idle device handles are reused
for repeated problem shapes."""
import numpy as np
import pytest

import synth

from _helpers import knots_of, problem_spec, max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MIX = [problem_spec(2, 2, (12, 9)), problem_spec(3, 2, (4, 5, 3)), problem_spec(2, 3, (8, 8), "RT"),
       problem_spec(2, 2, (12, 9)), problem_spec(3, 3, (3, 4, 4)), problem_spec(2, 4, (6, 10), "RT"),
       problem_spec(3, 2, (4, 5, 3)), problem_spec(2, 2, (12, 9))]


def _alone(spec, b, fd):
    disc = fd.TH if spec["disc"] == "TH" else fd.RT
    P = fd.Stokes(knots_of(spec), spec["p"], disc=disc, fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64)
    bt = torch.tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    info = P.solve(bt, x, tol=1e-8, maxit=800)[0]
    return x.cpu().numpy(), info


def _run(server, reqs, arrive_every=2):
    """Submit request k at step k * arrive_every; step until every request is done."""
    ids, step, max_active = [], 0, 0
    while True:
        while len(ids) < len(reqs) and len(ids) * arrive_every <= step:
            spec, b = reqs[len(ids)]
            disc = 0 if spec["disc"] == "TH" else 1
            ids.append(server.submit(knots_of(spec), spec["p"], b, float(step), disc=disc))
        active, queued, finished = server.step(float(step))
        max_active = max(max_active, active)
        step += 1
        if finished == len(reqs) and len(ids) == len(reqs):
            return ids, max_active
        assert step < 5000


def test_results_same_alone_and_in_the_mix():
    import paper_1712_00403_gb300 as fd
    reqs = []
    for k, spec in enumerate(MIX):
        from oracle import stokes as _s   # sizes only
        sizes = _s.build([synth.open_uniform_knots(nn, spec["p"]) for nn in spec["n_el"]], spec["p"],
                         spec["disc"]).block_sizes
        reqs.append((spec, synth.rhs(600 + k, sizes)))
    server = fd.Server(max_active=3, iters_per_step=3, fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64,
                       tol=1e-8, maxit=800)
    ids, max_active = _run(server, reqs)
    assert max_active <= 3
    st = server.stats()
    assert st["max_active_seen"] <= 3
    assert st["handles_reused"] >= 1          # repeated shapes come back to a cached handle
    for rid, (spec, b) in zip(ids, reqs):
        r = server.result(rid)
        assert r is not None and r["status"] == "OK" and r["true_rel_res"] <= 1e-8
        assert r["t_done"] >= r["t_admit"] >= r["t_arrival"]
        x1, info = _alone(spec, b, fd)
        assert abs(r["iterations"] - info["iterations"]) <= 1
        assert max_rel(r["x"], x1) <= 1e-7
        # the served solution solves the oracle's FP64 system
        S = _s.build(knots_of(spec), spec["p"], spec["disc"])
        res = np.linalg.norm(b - _s.matvec(S, r["x"])) / np.linalg.norm(b)
        assert res <= 1e-8, (spec, res)
    server.close()


def test_hbm_budget_limits_admission():
    """A budget of one and a half handles of a shape admits one request of that
    shape at a time (the idle handle is reused; a second one does not fit)."""
    import paper_1712_00403_gb300 as fd
    from oracle import stokes as _s
    spec = MIX[0]
    sizes = _s.build([synth.open_uniform_knots(nn, spec["p"]) for nn in spec["n_el"]], spec["p"],
                     spec["disc"]).block_sizes
    reqs = [(spec, synth.rhs(700 + k, sizes)) for k in range(4)]
    probe = fd.Server(max_active=8, iters_per_step=4, tol=1e-8, maxit=800)
    _run(probe, reqs[:1])
    one = probe.stats()["bytes_held"]          # one idle handle of this shape
    probe.close()
    assert one > 0
    server = fd.Server(max_active=8, hbm_budget_bytes=one + one // 2, iters_per_step=4, tol=1e-8, maxit=800)
    ids, max_active = _run(server, reqs, arrive_every=0)
    assert max_active == 1
    assert server.stats()["handles_created"] == 1
    for rid in ids:
        r = server.result(rid)
        assert r["status"] == "OK" and r["true_rel_res"] <= 1e-8
    server.close()
