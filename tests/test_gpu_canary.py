"""Guard-zone (canary) checks on every caller-owned output: the vectors handed
to the library are views into larger buffers whose leading and trailing
guard entries hold a fixed sentinel; after each call the guards must be
bit-for-bit unchanged. This catches stores past the ends of a block vector
(ragged tensor-core tiles, the last FP64 epilogue step, banded stencils at
the last row) that a comparison of the in-range values alone would miss."""
import numpy as np
import pytest

import synth

from _helpers import gpu_problem, problem_spec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G = 256                       # guard entries on each side (2 KB: keeps 16-byte alignment)
SENTINEL = 1.234567890123e300


def _guarded(n, fill=None):
    buf = torch.full((2 * G + n,), SENTINEL, dtype=torch.float64, device="cuda")
    view = buf[G:G + n]
    if fill is not None:
        view.copy_(fill)
    return buf, view


def _intact(buf):
    g = torch.cat([buf[:G], buf[-G:]]).cpu().numpy()
    return bool(np.all(g == SENTINEL))


@pytest.mark.parametrize("spec,fdp", [
    (problem_spec(3, 3, (5, 7, 9)), "tf32"),       # ragged row tiles and column tiles, three K stages
    (problem_spec(3, 3, (5, 7, 9)), "bf16"),
    (problem_spec(3, 3, (5, 7, 9)), "f64"),
    (problem_spec(2, 2, 140), "tf32"),             # n_v = 280: the column tile splits in two
    (problem_spec(2, 3, (8, 11), "RT"), "tf32"),
], ids=["3d-tf32", "3d-bf16", "3d-f64", "2d-280-tf32", "2d-rt-tf32"])
def test_apply_matvec_solve_stay_inside_their_vectors(spec, fdp):
    import paper_1712_00403_gb300 as fd
    prec = {"tf32": fd.FD_TF32X3, "bf16": fd.FD_BF16X6, "f64": fd.FD_F64}[fdp]
    nrhs = 3
    for mv in (fd.MV_F64, fd.MV_DF64):
        P = gpu_problem(spec, max_rhs=nrhs, fd_precision=prec, matvec_precision=mv)
        n = P.n_total * nrhs
        B = np.stack([synth.rhs(30 + j, P.block_sizes) for j in range(nrhs)]).reshape(-1)
        rb, r = _guarded(n, torch.tensor(B, device="cuda"))
        sb, s = _guarded(n)
        P.apply_prec(r, s)
        yb, y = _guarded(n)
        P.matvec(r, y)
        xb, x = _guarded(n, torch.zeros(n, dtype=torch.float64, device="cuda"))
        infos = P.solve(r, x, tol=1e-8, maxit=400)
        torch.cuda.synchronize()
        for name, buf in (("r", rb), ("s", sb), ("y", yb), ("x", xb)):
            assert _intact(buf), (name, mv)
        assert all(i["status"] == "OK" for i in infos)
        P.close()


def test_block_preconditioners_and_gmres_stay_inside_their_vectors():
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(problem_spec(3, 2, (4, 5, 6)), max_rhs=2, fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64)
    n = P.n_total * 2
    B = np.stack([synth.rhs(40 + j, P.block_sizes) for j in range(2)]).reshape(-1)
    rb, r = _guarded(n, torch.tensor(B, device="cuda"))
    for prec in (fd.PREC_PT, fd.PREC_PC):
        sb, s = _guarded(n)
        P.apply_block_prec(r, s, prec=prec)
        xb, x = _guarded(n, torch.zeros(n, dtype=torch.float64, device="cuda"))
        P.solve_gmres(r, x, prec=prec, tol=1e-8, maxit=300)
        torch.cuda.synchronize()
        assert _intact(sb) and _intact(xb) and _intact(rb)
