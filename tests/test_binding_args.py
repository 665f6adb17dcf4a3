"""CPU tests of the binding's argument checks: caller-supplied outputs and
host buffers are checked for type, dtype, place, layout and size before any
pointer reaches the library (it writes and copies exactly that many
elements)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1203_1269_gb300 import gp  # noqa: E402


def host_outs(T, **change):
    out = dict(nll=torch.empty(T, dtype=torch.float64), mu=torch.empty(T, dtype=torch.float64),
               sigma2=torch.empty(T, dtype=torch.float64), logdet=torch.empty(T, dtype=torch.float64),
               status=torch.empty(T, dtype=torch.int32))
    out.update(change)
    return out


REQ = ("nll", "mu", "sigma2", "status")


def test_valid_outputs_pass():
    out = host_outs(5)
    assert gp._check_outs(out, REQ, ("logdet",), 5, None) is out
    g = dict(nll=torch.empty(3, dtype=torch.float64), grad=torch.empty((3, 4), dtype=torch.float64),
             status=torch.empty(3, dtype=torch.int32))
    gp._check_outs(g, ("nll", "grad", "status"), (), 3, None, shapes={"grad": (3, 4)})


@pytest.mark.parametrize("change,err", [
    (dict(nll=torch.empty(4, dtype=torch.float64)), ValueError),           # too short
    (dict(mu=torch.empty(6, dtype=torch.float64)), ValueError),            # too long
    (dict(sigma2=torch.empty(5, dtype=torch.float32)), TypeError),         # wrong dtype
    (dict(status=torch.empty(5, dtype=torch.int64)), TypeError),           # status must be int32
    (dict(logdet=torch.empty(10, dtype=torch.float64)[::2]), ValueError),  # not contiguous
    (dict(nll=[0.0] * 5), TypeError),                                      # not a tensor
    (dict(nll=None), ValueError),                                          # required key missing
])
def test_bad_outputs_rejected(change, err):
    with pytest.raises(err):
        gp._check_outs(host_outs(5, **change), REQ, ("logdet",), 5, None)


def test_grad_shape_checked():
    g = dict(nll=torch.empty(3, dtype=torch.float64), grad=torch.empty((3, 5), dtype=torch.float64),
             status=torch.empty(3, dtype=torch.int32))
    with pytest.raises(ValueError):
        gp._check_outs(g, ("nll", "grad", "status"), (), 3, None, shapes={"grad": (3, 4)})


def test_host_batch_args():
    x = torch.zeros((10, 3), dtype=torch.float64)
    y = torch.zeros(10, dtype=torch.float64)
    th = torch.ones((4, 3), dtype=torch.float64)
    assert gp._host_batch_args(x, y, th) == (10, 3, 4)
    with pytest.raises(ValueError):
        gp._host_batch_args(x, torch.zeros(9, dtype=torch.float64), th)     # y shorter than n
    with pytest.raises(ValueError):
        gp._host_batch_args(x, y, torch.ones((4, 2), dtype=torch.float64))  # theta rows of d - 1
    with pytest.raises(ValueError):
        gp._host_batch_args(x.float(), y, th)                              # not float64
    with pytest.raises(ValueError):
        gp._host_batch_args(torch.zeros(10, dtype=torch.float64), y, th)   # x not 2-D
