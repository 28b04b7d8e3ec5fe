"""Split-TF32 and split-BF16 tcgen05 FD applies vs. the FP64 oracle, through
the C ABI.

Bar: element-wise relative error max|s - s_ref| / max|s_ref| of every block
<= 1e-5 (split-TF32: three TF32
products; split-BF16: three bf16 pieces per operand and the six leading
products; FP32 accumulation and FP32 intermediates in both); P_D-MINRES with
either apply reaches the true relative residual 1e-8 within 2 iterations of
the FP64 run.
"""
import numpy as np
import pytest

import synth
from oracle import stokes

from _helpers import gpu_problem, oracle_problem, problem_spec, max_rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    problem_spec(3, 2, 4),
    problem_spec(3, 3, (3, 4, 6)),
    problem_spec(3, 3, 9),             # 27 interior functions: rows span several 128-row tiles
    problem_spec(3, 2, 40),            # n = 80 per direction, three K stages, N padded to 80
    problem_spec(2, 2, 16),
    problem_spec(2, 3, 70),            # n = 141 > 128: N tile of 144, ragged K stage
    problem_spec(2, 2, 6, "RT"),
    problem_spec(2, 2, 140),           # n = 280 > 256: the N tile splits in two, ragged second half
    problem_spec(3, 6, (90, 17, 23)),  # a batched-workload-sized instance: p = 6, n = 184 x 38 x 50
    problem_spec(3, 1, (1, 2, 3)),     # degenerate: a direction with one function (K = N = 1)
    problem_spec(2, 5, 1),             # one element at p = 5
]


def _ids(c):
    return f"{c['disc']}-d{c['dim']}-p{c['p']}-{'x'.join(map(str, c['n_el']))}"


@pytest.mark.parametrize("split", ["tf32", "bf16"])
@pytest.mark.parametrize("spec", CASES, ids=_ids)
def test_tf32_apply_matches_oracle(spec, split):
    import paper_1712_00403_gb300 as fd
    P = gpu_problem(spec, max_rhs=2, fd_precision=fd.FD_TF32X3 if split == "tf32" else fd.FD_BF16X6)
    S = oracle_problem(spec)
    R = np.stack([synth.random_vector(500 + j, P.n_total) for j in range(2)])
    r = torch.tensor(R.reshape(-1), device="cuda")
    s = torch.empty_like(r)
    P.apply_prec(r, s)
    out = s.cpu().numpy().reshape(2, -1)
    assert fd.device_error() == 0
    for j in range(2):
        ref = stokes.apply_PD_inv(S, R[j], "fd")
        for o0, o1 in zip(P.block_offsets[:-1], P.block_offsets[1:]):
            assert max_rel(out[j, o0:o1], ref[o0:o1]) <= 1e-5


@pytest.mark.parametrize("split", ["tf32", "bf16"])
@pytest.mark.parametrize("spec", [problem_spec(3, 2, 6), problem_spec(2, 2, 16)], ids=_ids)
def test_tf32_minres_within_two_iterations_of_f64(spec, split):
    import paper_1712_00403_gb300 as fd
    P32 = gpu_problem(spec, max_rhs=2, fd_precision=fd.FD_TF32X3 if split == "tf32" else fd.FD_BF16X6)
    P64 = gpu_problem(spec, max_rhs=2, fd_precision=fd.FD_F64)
    B = np.stack([synth.rhs(60 + j, P32.block_sizes) for j in range(2)])
    b = torch.tensor(B.reshape(-1), device="cuda")
    x32, x64 = torch.zeros_like(b), torch.zeros_like(b)
    i32 = P32.solve(b, x32, tol=1e-8, maxit=500)
    i64 = P64.solve(b, x64, tol=1e-8, maxit=500)
    for a, c in zip(i32, i64):
        assert a["status"] == "OK" and a["true_rel_res"] <= 1e-8
        assert a["iterations"] <= c["iterations"] + 2
    assert fd.device_error() == 0
