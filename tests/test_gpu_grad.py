"""Gradient of -2logL with respect to theta (gp_nll_grad_batch) against the
oracle, and at full size against central differences of the GPU's own
double-precision -2logL."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
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


@pytest.mark.parametrize("corr,p", [("powexp", 1.95), ("powexp", 1.0), ("matern12", 2.0), ("matern32", 2.0), ("matern52", 2.0)])
def test_grad_matches_oracle(ctx, corr, p):
    g = np.random.default_rng(61)
    n, d, T, delta = 300, 3, 5, 1e-4
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, T, d, lo=0.0, hi=1.2)
    try:
        ctx.set_options(correlation=corr)
        res = ctx.nll_grad_batch(dev(x), dev(y), dev(th), p, delta)
        plain = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "fp64")
    finally:
        ctx.set_options(correlation="powexp")
    assert np.all(host(res["status"]) == 0)
    # the likelihood comes from the same kernels as gp_nll_batch
    assert np.array_equal(host(res["nll"]), host(plain["nll"]))
    G = host(res["grad"])
    worst = 0.0
    for t in range(T):
        go, out, st = oracle.nll_grad(x, y, th[t], p, delta, corr=corr)
        assert st == 0
        err = np.max(np.abs(G[t] - go)) / max(np.max(np.abs(go)), 1.0)
        worst = max(worst, err)
    print(f"\n{corr} p={p}: gradient max rel err {worst:.2e}")
    assert worst <= 1e-8


def test_grad_status_rows(ctx):
    """A candidate whose R is numerically singular (nearly constant
    correlation, no nugget) fails with a status and a NaN gradient row; the
    other candidate of the same batch is unaffected."""
    g = np.random.default_rng(62)
    x = g.random((140, 2))
    y = x[:, 0] + np.sin(5 * x[:, 1])
    th = np.array([[1e-3, 1e-3], [100.0, 100.0]])
    res = ctx.nll_grad_batch(dev(x), dev(y), dev(th), 2.0, 0.0)
    st = host(res["status"])
    G = host(res["grad"])
    ref, st1 = oracle.nll_batch(x, y, th, 2.0, 0.0)
    assert st1[0] != 0 and st1[1] == 0
    assert st[0] != 0 and np.all(np.isnan(G[0]))
    assert st[1] == 0 and np.all(np.isfinite(G[1]))
    go, _, _ = oracle.nll_grad(x, y, th[1], 2.0, 0.0)
    assert np.max(np.abs(G[1] - go)) <= 1e-8 * max(np.max(np.abs(go)), 1.0)


def test_grad_full_size_finite_differences(ctx):
    """n = 4000, d = 6 (the multi-start workload's design): the gradient
    against central differences of the GPU's own double-precision -2logL, a
    property that holds at any size."""
    w = inputs.hartman_shape()
    g = np.random.default_rng(63)
    sample = inputs.log_uniform_thetas(g, 3, w.d, lo=-0.3, hi=0.7)   # cond(R) small enough for differences
    res = ctx.nll_grad_batch(dev(w.x), dev(w.y), dev(sample), w.p, w.delta)
    assert np.all(host(res["status"]) == 0)
    G = host(res["grad"])
    pts, hs = [], []
    for t in range(len(sample)):
        for k in range(w.d):
            h = 1e-5 * sample[t, k]
            for s_ in (1.0, -1.0):
                q = sample[t].copy()
                q[k] += s_ * h
                pts.append(q)
            hs.append(h)
    f = host(ctx.nll_batch(dev(w.x), dev(w.y), dev(np.array(pts)), w.p, w.delta, "fp64")["nll"])
    fd = ((f[0::2] - f[1::2]) / (2 * np.array(hs))).reshape(len(sample), w.d)
    rel = np.abs(G - fd) / np.maximum(np.abs(fd), 1.0)
    print(f"\nn=4000 d=6: |grad| up to {np.abs(G).max():.3e}, max rel diff to central differences {rel.max():.2e}")
    assert rel.max() <= 1e-4


def test_grad_chunked_matches_one_chunk(ctx):
    g = np.random.default_rng(64)
    x = inputs.random_lhd(g, 260, 2)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, 5, 2, lo=0.0, hi=1.0)
    base = ctx.options()
    try:
        ref = ctx.nll_grad_batch(dev(x), dev(y), dev(th), 1.95, 1e-5)
        ctx.set_options(max_batch=2)
        got = ctx.nll_grad_batch(dev(x), dev(y), dev(th), 1.95, 1e-5)
    finally:
        ctx.set_options(**base)
    for k in ("nll", "grad", "status"):
        assert np.array_equal(host(got[k]), host(ref[k]), equal_nan=True), k



def test_grad_at_max_d(ctx):
    """d = 16, the largest d the gradient is built for, against the oracle;
    d = 17 is refused with GP_ENOTSUP."""
    from paper_1203_1269_gb300 import gp
    g = np.random.default_rng(65)
    n, d, delta = 200, 16, 1e-6
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, 2, d, lo=-1.0, hi=0.0)
    res = ctx.nll_grad_batch(dev(x), dev(y), dev(th), 1.95, delta)
    assert np.all(host(res["status"]) == 0)
    G = host(res["grad"])
    for t in range(len(th)):
        go, _, st = oracle.nll_grad(x, y, th[t], 1.95, delta)
        assert st == 0
        assert np.max(np.abs(G[t] - go)) <= 1e-8 * max(np.max(np.abs(go)), 1.0)
    x17 = g.random((n, 17))
    with pytest.raises(gp.GPError) as e:
        ctx.nll_grad_batch(dev(x17), dev(y), dev(g.random((1, 17))), 1.95, delta)
    assert e.value.code == gp.GP_ENOTSUP
