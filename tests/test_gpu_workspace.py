"""gp_call_bytes against what the calls allocate on the device: on a fresh
context (empty arena) the workspace after a call is the reported figure, and
a model holds exactly the reported bytes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1203_1269_gb300 import inputs

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp as gp_mod
    return gp_mod


@pytest.fixture(scope="module")
def problem():
    g = np.random.default_rng(71)
    x = inputs.random_lhd(g, 300, 3)
    return x, inputs.y_sinsum(x), inputs.log_uniform_thetas(g, 5, 3, lo=0.0, hi=1.0)


@pytest.mark.parametrize("prec", ["mixed", "fp32", "fp64", "auto"])
def test_nll_batch_workspace(gp, problem, prec):
    x, y, th = problem
    ctx = gp.Context(0)
    try:
        want = ctx.call_bytes("nll_batch", 300, 3, len(th), prec)
        ctx.nll_batch(dev(x), dev(y), dev(th), 1.95, 1e-6, prec)
        torch.cuda.synchronize()
        got = ctx.workspace_bytes()
    finally:
        ctx.close()
    if prec == "auto":
        assert 0 < got <= want      # an upper bound: the tiers it reached, routing buffers apart
    else:
        assert got == want


def test_grad_workspace(gp, problem):
    x, y, th = problem
    ctx = gp.Context(0)
    try:
        want = ctx.call_bytes("nll_grad", 300, 3, len(th))
        ctx.nll_grad_batch(dev(x), dev(y), dev(th), 1.95, 1e-6)
        torch.cuda.synchronize()
        assert ctx.workspace_bytes() == want
    finally:
        ctx.close()


def test_fit_and_predict_bytes(gp, problem):
    x, y, th = problem
    ctx = gp.Context(0)
    try:
        want_fit = ctx.call_bytes("fit", 300, 3)
        model = ctx.fit(dev(x), dev(y), dev(th[0]), 1.95, 1e-6)
        assert model.bytes == want_fit
        N = 700
        want_pred = ctx.call_bytes("predict", 300, 3, N)
        ctx.predict(model, dev(inputs.uniform_design(inputs.rng(72), N, 3)))
        torch.cuda.synchronize()
        assert ctx.workspace_bytes() == want_pred
        model.free()
    finally:
        ctx.close()
