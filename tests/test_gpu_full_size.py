"""Parity at the full size of the 3D cube workload (Taylor-Hood, p=3, 64^3
elements, 6,740,830 unknowns, 16 right-hand sides) in the configuration the
benchmark times: split-TF32 FD apply, double-float matvec, 16 right-hand
sides per call. Whole vectors of the first and the last right-hand side are
compared with the oracle (its FP64 Kronecker matvec and FD apply take a few
seconds each at this size): the matvec within 1e-12 and the apply within 1e-5
per block; the solve ends with status OK and an FP64 true residual <= 1e-8 for
every right-hand side, confirmed for the first and the last with the oracle's
own matvec."""
import numpy as np
import pytest

import synth
from oracle import stokes

from _helpers import max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRHS = 16
SEEDS = list(range(200, 200 + NRHS))


@pytest.fixture(scope="module")
def cube():
    import paper_1712_00403_gb300 as fd
    knots = synth.knots_for("cube_th_p3_64")
    S = stokes.build(knots, 3)
    P = fd.Stokes(knots, 3, fd_precision=fd.FD_TF32X3, max_rhs=NRHS, matvec_precision=fd.MV_DF64)
    assert P.n_total == S.n_total == 6_740_830
    B = np.stack([synth.rhs(s, P.block_sizes) for s in SEEDS])
    yield S, P, B
    P.close()


def _blocks(P, a, b):
    return [max_rel(a[o0:o1], b[o0:o1]) for o0, o1 in zip(P.block_offsets[:-1], P.block_offsets[1:])]


def test_full_size_matvec_and_apply(cube):
    S, P, B = cube
    x = torch.tensor(B.reshape(-1), device="cuda")
    y = torch.empty_like(x)
    s = torch.empty_like(x)
    P.matvec(x, y)
    P.apply_prec(x, s)
    torch.cuda.synchronize()
    n = P.n_total
    for j in (0, NRHS - 1):
        yj = y[j * n:(j + 1) * n].cpu().numpy()
        sj = s[j * n:(j + 1) * n].cpu().numpy()
        assert max(_blocks(P, yj, stokes.matvec(S, B[j]))) <= 1e-12
        assert max(_blocks(P, sj, stokes.apply_PD_inv(S, B[j]))) <= 1e-5


def test_full_size_solve(cube):
    S, P, B = cube
    b = torch.tensor(B.reshape(-1), device="cuda")
    x = torch.zeros_like(b)
    infos = P.solve(b, x, tol=1e-8, maxit=400)
    assert len(infos) == NRHS
    for info in infos:
        assert info["status"] == "OK" and info["true_rel_res"] <= 1e-8, info
    n = P.n_total
    for j in (0, NRHS - 1):
        xj = x[j * n:(j + 1) * n].cpu().numpy()
        assert np.linalg.norm(B[j] - stokes.matvec(S, xj)) <= 1.01e-8 * np.linalg.norm(B[j])
