"""Batches recorded as CUDA graphs (gp_plan_nll_batch / gp_plan_launch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1203_1269_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    return gp.Context(0)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


KEYS = ("nll", "mu", "sigma2", "logdet", "status")


@pytest.mark.parametrize("prec,cond", [("mixed", False), ("fp64", False), ("fp32", True), ("mixed", True)])
def test_plan_replays_the_call(ctx, prec, cond):
    g = np.random.default_rng(501)
    n, d, T, p, delta = 389, 3, 12, 1.95, 1e-6
    x = dev(inputs.random_lhd(g, n, d))
    y = dev(inputs.y_sinsum(host(x)))
    th = dev(inputs.log_uniform_thetas(g, T, d, lo=-0.5, hi=1.0))
    l0 = ctx.launch_count()
    direct = ctx.nll_batch(x, y, th, p, delta, prec, cond=cond)
    torch.cuda.synchronize()
    per_call = ctx.launch_count() - l0
    plan = ctx.plan_nll_batch(x, y, th, p, delta, prec, cond=cond)
    assert plan.kernels == per_call
    keys = KEYS + (("cond",) if cond else ())
    for k in keys:                                  # the eager evaluation at creation
        assert np.array_equal(host(plan.out[k]), host(direct[k]), equal_nan=True)
    for k in keys:
        plan.out[k].fill_(0)
    l1 = ctx.launch_count()
    plan.launch()
    torch.cuda.synchronize()
    assert ctx.launch_count() - l1 == plan.kernels
    for k in keys:
        assert np.array_equal(host(plan.out[k]), host(direct[k]), equal_nan=True)
    # a replay reads the bound tensors' current contents
    th.copy_(dev(inputs.log_uniform_thetas(g, T, d, lo=-0.5, hi=1.0)))
    plan.launch()
    again = ctx.nll_batch(x, y, th, p, delta, prec, cond=cond)
    torch.cuda.synchronize()
    for k in keys:
        assert np.array_equal(host(plan.out[k]), host(again[k]), equal_nan=True)
    plan.free()


def test_plan_of_a_chunked_batch(ctx):
    """A batch processed in chunks (max_batch = 4 of T = 10) records every
    chunk's launches in the graph and replays to the same bits."""
    g = np.random.default_rng(503)
    x = dev(inputs.random_lhd(g, 300, 3))
    y = dev(inputs.y_sinsum(host(x)))
    th = dev(inputs.log_uniform_thetas(g, 10, 3, lo=-0.5, hi=1.0))
    base = ctx.options()
    try:
        ctx.set_options(max_batch=4)
        l0 = ctx.launch_count()
        direct = ctx.nll_batch(x, y, th, 1.95, 1e-6, "mixed")
        torch.cuda.synchronize()
        per_call = ctx.launch_count() - l0
        plan = ctx.plan_nll_batch(x, y, th, 1.95, 1e-6, "mixed")
    finally:
        ctx.set_options(**base)
    assert plan.kernels == per_call
    for k in KEYS:
        plan.out[k].fill_(0)
    plan.launch()
    torch.cuda.synchronize()
    for k in KEYS:
        assert np.array_equal(host(plan.out[k]), host(direct[k]), equal_nan=True), k
    plan.free()


def test_plan_owns_its_workspace(ctx):
    """Calls that regrow the context's workspace leave the plan intact."""
    g = np.random.default_rng(502)
    x = dev(inputs.random_lhd(g, 200, 2))
    y = dev(inputs.y_sinsum(host(x)))
    th = dev(inputs.log_uniform_thetas(g, 8, 2))
    plan = ctx.plan_nll_batch(x, y, th, 2.0, 1e-6, "mixed")
    ref = {k: host(plan.out[k]).copy() for k in KEYS}
    assert plan.bytes > 0
    xb = dev(inputs.random_lhd(g, 1500, 2))
    ctx.nll_batch(xb, dev(inputs.y_sinsum(host(xb))), dev(inputs.log_uniform_thetas(g, 64, 2)), 2.0, 1e-6, "mixed")
    plan.launch()
    torch.cuda.synchronize()
    for k in KEYS:
        assert np.array_equal(host(plan.out[k]), ref[k], equal_nan=True)
    plan.free()


def test_plan_rejects_auto_and_outlives_context():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    c = gp.Context(0)
    w = inputs.small_grid_fit()
    x, y, th = dev(w.x), dev(w.y), dev(w.thetas[:4])
    with pytest.raises(gp.GPError) as e:
        c.plan_nll_batch(x, y, th, w.p, w.delta, "auto")
    assert e.value.code == gp.GP_ENOTSUP
    plan = c.plan_nll_batch(x, y, th, w.p, w.delta, "fp64")
    c.close()
    with pytest.raises(gp.GPError):
        plan.launch()
    plan.free()
