"""fdst_fd_apply_static: the allocation-free FD block solve for callers that
cannot call cudaMalloc (it keeps its scratch in a fixed file-scope device
array). Checked through the C ABI against the existing fdst_apply_prec on two
consecutive calls, with the 1e-12 tolerance of the FP64 parity tests, and at
the static array's limits against a host FP64 evaluation of the same
definition. Collected last so that a failure here does not hide any other test."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import stokes, univariate as uv

from _helpers import gpu_problem, max_rel, oracle_problem, problem_spec

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
        assert max_rel(s_blk.cpu().numpy(), s_full[o0:o1].cpu().numpy()) <= 1e-12


def _host_fd(U, lam, coef, r):
    """s = (U_d x .. x U_1) Delta^{-1} (U_d x .. x U_1)^T r in FP64 on the host,
    with Delta = sum_d coef_d lam_d and index 1 fastest."""
    dim = len(U)
    shape = [u.shape[0] for u in U][::-1]           # C order: slowest direction first
    x = r.reshape(shape)
    for d in range(dim):
        x = np.moveaxis(np.tensordot(U[d].T, x, axes=([1], [dim - 1 - d])), 0, dim - 1 - d)
    delta = np.zeros(shape)
    for d in range(dim):
        sh = [1] * dim
        sh[dim - 1 - d] = -1
        delta = delta + coef[d] * lam[d].reshape(sh)
    x = x / delta
    for d in range(dim):
        x = np.moveaxis(np.tensordot(U[d], x, axes=([1], [dim - 1 - d])), 0, dim - 1 - d)
    return x.reshape(-1)


def test_static_apply_at_its_limits_allocates_nothing():
    """At the documented limits (n_d = 256, and 256 x 96 x 96 = 2,359,296
    entries, the full intermediate slice) the result matches a host FP64
    evaluation, on two calls in a row, and a warm call leaves the device's
    free memory unchanged."""
    import paper_1712_00403_gb300 as fd
    cases = [(2, [128, 128]), (3, [128, 48, 48])]      # spline pencils: n_v = 2 n_el + p - 2 with p = 2
    for call, (dim, n_el) in enumerate(cases):
        spaces = [uv.interior_space(synth_knots(n), 3) for n in n_el]
        Uh, lamh = [], []
        for sp in spaces:
            l, u = sla.eigh(uv.stiffness(sp), uv.mass(sp))
            Uh.append(np.ascontiguousarray(u))
            lamh.append(l)
        coef = [2.0] + [1.0] * (dim - 1)
        N = int(np.prod([u.shape[0] for u in Uh]))
        assert [u.shape[0] for u in Uh][0] == 256
        r_h = synth.random_vector(950 + call, N)
        ref = _host_fd(Uh, lamh, coef, r_h)
        U = [torch.tensor(u, device="cuda") for u in Uh]
        lam = [torch.tensor(l, device="cuda") for l in lamh]
        r = torch.tensor(r_h, device="cuda")
        s = torch.full_like(r, float("nan"))
        fd.fd_apply_static(U, lam, coef, r, s)            # warm call
        torch.cuda.synchronize()
        assert max_rel(s.cpu().numpy(), ref) <= 1e-12
        free0 = torch.cuda.mem_get_info()[0]
        s.fill_(float("nan"))
        fd.fd_apply_static(U, lam, coef, r, s)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (free0, free1)
        assert max_rel(s.cpu().numpy(), ref) <= 1e-12


def synth_knots(n_el):
    """Velocity knot vector of the TH space at p = 2 (degree 3, interior knots doubled)."""
    from oracle import splines
    return splines.elevate_knots(synth.open_uniform_knots(n_el, 2), 2)


def test_static_apply_rejects_oversized_and_overlapping_buffers():
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
    # r and s overlapping by part of their length
    k = 8
    Uk = [torch.eye(k, dtype=torch.float64, device="cuda")] * 2
    lk = [torch.ones(k, dtype=torch.float64, device="cuda")] * 2
    buf = torch.ones(k * k + 5, dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FdstError) as e:
        fd.fd_apply_static(Uk, lk, [1.0, 1.0], buf[:k * k], buf[5:])
    assert "overlap" in str(e.value)
