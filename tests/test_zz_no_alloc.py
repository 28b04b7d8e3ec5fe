"""fdst_fd_apply_static: the allocation-free FD block solve for callers that
cannot call cudaMalloc (it keeps its scratch in a fixed file-scope device
array). Checked through the C ABI against the existing fdst_apply_prec on two
consecutive calls, with the 1e-12 tolerance of the FP64 parity tests.
Collected last so that a failure here does not hide any other test."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import stokes

from _helpers import gpu_problem, oracle_problem, problem_spec, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _factors(S, k):
    """U_d, lam_d of the pencils of velocity component k (LAPACK, as inputs)."""
    Ks, Ms, coef = stokes.pv_pencils(S, k)
    U, lam = [], []
    for K, M in zip(Ks, Ms):
        l, u = sla.eigh(K, M)
        U.append(torch.tensor(np.ascontiguousarray(u), device="cuda"))
        lam.append(torch.tensor(l, device="cuda"))
    return U, lam, coef


@pytest.mark.parametrize("spec", [problem_spec(3, 2, (4, 5, 6)), problem_spec(2, 3, (7, 5))],
                         ids=["3d-4x5x6", "2d-7x5"])
def test_static_apply_matches_apply_prec_twice(spec):
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(spec, max_rhs=1)
    S = oracle_problem(spec)
    # two calls in a row on different blocks / right-hand sides share the static scratch
    for call, k in enumerate((0, 1)):
        r_full = torch.tensor(synth.random_vector(900 + call, P.n_total), device="cuda")
        s_full = torch.empty_like(r_full)
        P.apply_prec(r_full, s_full)
        o0, o1 = P.block_offsets[k], P.block_offsets[k + 1]
        U, lam, coef = _factors(S, k)
        r_blk = r_full[o0:o1].contiguous()
        s_blk = torch.full_like(r_blk, float("nan"))
        fd.fd_apply_static(U, lam, coef, r_blk, s_blk)
        torch.cuda.synchronize()
        assert rel(s_blk.cpu().numpy(), s_full[o0:o1].cpu().numpy()) <= 1e-12


def test_static_apply_rejects_oversized_blocks():
    import paper_1712_00403_gb300 as fd
    n = 300                                            # > 256 per direction
    U = [torch.eye(n, dtype=torch.float64, device="cuda")] * 2
    lam = [torch.ones(n, dtype=torch.float64, device="cuda")] * 2
    r = torch.ones(n * n, dtype=torch.float64, device="cuda")
    s = torch.empty_like(r)
    with pytest.raises(fd.FdstError) as e:
        fd.fd_apply_static(U, lam, [1.0, 1.0], r, s)
    assert "256" in str(e.value)
    m = 140                                            # 140^3 > 2359296 entries
    U3 = [torch.eye(m, dtype=torch.float64, device="cuda")] * 3
    lam3 = [torch.ones(m, dtype=torch.float64, device="cuda")] * 3
    r3 = torch.ones(m ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FdstError) as e:
        fd.fd_apply_static(U3, lam3, [1.0, 1.0, 2.0], r3, torch.empty_like(r3))
    assert "static maximum" in str(e.value)
