"""CPU tests: the binding checks every size the C entry points cannot see
before any call reaches the library (no GPU is touched)."""
import pytest

torch = pytest.importorskip("torch")

import paper_1712_00403_gb300 as fd  # noqa: E402


def _t(*shape):
    return torch.zeros(*shape, dtype=torch.float64)


@pytest.mark.parametrize("U,lam,coef,r,s,msg", [
    ([_t(4, 4)], [_t(4)], [1.0], _t(4), _t(4), "2 or 3 directions"),
    ([_t(4, 4)] * 4, [_t(4)] * 4, [1.0] * 4, _t(256), _t(256), "2 or 3 directions"),
    ([_t(4, 4)] * 3, [_t(4)] * 3, [1.0, 1.0], _t(64), _t(64), "coefficients"),
    ([_t(4, 4)] * 3, [_t(4)] * 2, [1.0] * 3, _t(64), _t(64), "eigenvalue vectors"),
    ([_t(4, 5), _t(4, 4)], [_t(4)] * 2, [1.0] * 2, _t(16), _t(16), "square"),
    ([_t(4, 4), _t(3, 3)], [_t(4), _t(4)], [1.0] * 2, _t(12), _t(12), "lam_2"),
    ([_t(4, 4), _t(3, 3)], [_t(4), _t(3)], [1.0] * 2, _t(11), _t(12), "r has 11"),
    ([_t(4, 4), _t(3, 3)], [_t(4), _t(3)], [1.0] * 2, _t(12), _t(13), "s has 13"),
])
def test_fd_apply_static_rejects_bad_sizes(U, lam, coef, r, s, msg):
    with pytest.raises(ValueError) as e:
        fd.fd_apply_static(U, lam, coef, r, s)
    assert msg in str(e.value)


def test_fd_apply_static_rejects_host_tensors_of_the_right_size():
    with pytest.raises(TypeError):
        fd.fd_apply_static([_t(4, 4), _t(3, 3)], [_t(4), _t(3)], [1.0, 1.0], _t(12), _t(12))
