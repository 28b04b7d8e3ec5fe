"""Failure detection without a GPU fault: every spin wait of the tensor-core
kernel is bounded (about 2 s of the global timer) and reports expiry instead of
hanging. A self-test kernel waits, through that same bounded wait, on an
mbarrier nothing arrives on; it must give up, raise its abort flag and return,
and the device must stay usable (a solve afterwards reaches the tolerance)."""
import pytest

import synth

from _helpers import gpu_problem, problem_spec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_expires_and_device_stays_usable():
    import paper_1712_00403_gb300 as fd
    status, gave_up, seconds = fd.check_bounded_wait()
    assert status == "TIMEOUT" and gave_up
    assert 1.5 <= seconds <= 20.0
    assert fd.device_error() == 0          # the contraction kernel's flag is untouched
    P = gpu_problem(problem_spec(2, 2, 8), fd_precision=fd.FD_TF32X3)
    b = torch.tensor(synth.rhs(9, P.block_sizes), device="cuda")
    x = torch.zeros_like(b)
    info = P.solve(b, x, tol=1e-8, maxit=300)[0]
    assert info["status"] == "OK" and info["true_rel_res"] <= 1e-8
