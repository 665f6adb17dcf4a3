"""Kriging variances with v = L^-1 r on the tensor cores (predict_tc = 1,
the default) against the oracle and against the double-float substitution
on the FP32 pipes (predict_tc = 0) on the same model.

Tolerances: s2 within 1e-8 sigma2_hat of the oracle (the FP64 path's
prediction tolerance, where cond(R) <= 1e8); between the two GPU paths
within 2e-9 sigma2_hat -- a CPU emulation of the tensor-core arithmetic
(5 slices in the updates, 7 in the diagonal steps, one fixed exponent for
v) against an FP64 substitution gave 5e-11 .. 4e-10 sigma2_hat at n = 2048
and cond(R) up to 5e8.  Means: r'w in double-float on both paths, within
1e-8 of the oracle relative to max |yhat|.
"""
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
    c = gp.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.cpu().numpy()


def both_paths(ctx, model, xs, want_var=True):
    out = {}
    for tc in (1, 0):
        ctx.set_options(predict_tc=tc)
        yh, s2 = ctx.predict(model, dev(xs), want_var=want_var)
        out[tc] = (host(yh), None if s2 is None else host(s2))
    ctx.set_options(predict_tc=1)
    return out


# (n, d, N, p, delta, theta scale): ragged n (one tile row, several, a
# ragged last one), ragged N (one point, a partial block, several blocks), a
# large nugget (|v_i|^2 <= 1 + delta = 4: the slices of v take exponent 2),
# p below 1
CASES = [(1, 2, 5, 1.95, 1e-6, 1.0), (100, 3, 129, 1.95, 1e-8, 4.0), (129, 1, 1, 2.0, 1e-6, 20.0),
         (260, 3, 300, 1.95, 0.0, 4.0), (700, 6, 257, 1.9, 1e-6, 1.0), (1100, 4, 64, 2.0, 1e-6, 2.0),
         (400, 2, 200, 2.0, 3.0, 2.0), (300, 3, 150, 0.7, 1e-6, 2.0)]


@pytest.mark.parametrize("n,d,N,p,delta,ts", CASES)
def test_tc_variance_matches_oracle_and_fp32_path(ctx, n, d, N, p, delta, ts):
    g = np.random.default_rng(1000 + n + d)
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    theta = ts * (0.5 + g.random(d))
    model = ctx.fit(dev(x), dev(y), dev(theta), p, delta, "fp64")
    xs = np.vstack([x[: min(n, N // 3)], g.random((N - min(n, N // 3), d))])
    res = both_paths(ctx, model, xs)
    (y1, s1), (y0, s0) = res[1], res[0]
    yo, so, st = oracle.predict(x, y, theta, p, delta, xs)
    assert st == 0
    sig = model.sigma2
    scale = max(1.0, np.max(np.abs(yo)))
    assert np.all(np.isfinite(s1))
    assert np.max(np.abs(y1 - yo)) <= 1e-8 * scale
    assert np.max(np.abs(s1 - so)) <= 1e-8 * sig + 1e-14
    assert np.max(np.abs(s1 - s0)) <= 2e-9 * sig + 1e-14, np.max(np.abs(s1 - s0)) / sig
    assert np.max(np.abs(y1 - y0)) <= 1e-9 * scale
    # yhat: the same bits without variances
    y2, none = ctx.predict(model, dev(xs), want_var=False)
    assert none is None and np.array_equal(host(y2), y1)
    model.free()


def test_tc_ill_conditioned_against_fp32_path(ctx):
    """cond(R) ~ 1e8 (d = 6, p = 2, small theta, n = 1500): the two GPU
    paths within 2e-9 sigma2_hat, the oracle within its own rounding bound
    (the FP64 path's parity tests allow n cond u beyond 1e8)."""
    g = np.random.default_rng(77)
    n, d, N = 1500, 6, 400
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_bump(x)
    theta = np.full(d, 1.5)
    o, st = oracle.nll(x, y, theta, 2.0, 1e-6, want_cond=True)
    assert st == 0
    model = ctx.fit(dev(x), dev(y), dev(theta), 2.0, 1e-6, "fp64")
    xs = g.random((N, d))
    res = both_paths(ctx, model, xs)
    sig = model.sigma2
    d01 = np.max(np.abs(res[1][1] - res[0][1])) / sig
    print(f"\ncond1 {o['cond1']:.2e}: max |s2_tc - s2_fp32| / sigma2 = {d01:.2e}")
    assert d01 <= 2e-9
    yo, so, _ = oracle.predict(x, y, theta, 2.0, 1e-6, xs)
    bound = max(1e-8, n * o["cond1"] * 2.0 ** -53)
    assert np.max(np.abs(res[1][1] - so)) <= bound * sig


def test_tc_split_model_and_matern(ctx):
    """A split-precision fit and a Matern 5/2 fit: the same parity on the
    tensor-core path."""
    g = np.random.default_rng(5)
    n, d, N = 900, 4, 300
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    theta = np.array([3.0, 1.0, 2.0, 5.0])
    for prec, corr in (("mixed", "powexp"), ("fp64", "matern52")):
        ctx.set_options(correlation=corr)
        try:
            model = ctx.fit(dev(x), dev(y), dev(theta), 1.95, 1e-6, prec)
        finally:
            ctx.set_options(correlation="powexp")
        xs = g.random((N, d))
        res = both_paths(ctx, model, xs)
        sig = model.sigma2
        assert np.max(np.abs(res[1][1] - res[0][1])) <= 2e-9 * sig
        yo, so, _ = oracle.predict(x, y, theta, 1.95, 1e-6, xs, corr=corr)
        tol = 1e-8 if prec == "fp64" else 1e-6
        assert np.max(np.abs(res[1][1] - so)) <= tol * sig, (prec, corr)
        model.free()


def test_tc_chunks_give_the_same_bits():
    """A budget that leaves room for one point block per chunk runs many
    chunks of one CTA each: the same bits as the default one-wave chunks."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    g = np.random.default_rng(12)
    n, d, N = 300, 3, 1000
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    theta = np.array([2.0, 4.0, 3.0])
    xs = g.random((N, d))
    out = []
    for budget in (0, 4 << 20):
        c = gp.Context(0, hbm_budget_bytes=budget)
        try:
            model = c.fit(dev(x), dev(y), dev(theta), 1.95, 1e-8, "fp64")
            before = c.launch_count()
            yh, s2 = c.predict(model, dev(xs))
            out.append((host(yh), host(s2), c.launch_count() - before))
            model.free()
        finally:
            c.close()
    (y0, v0, l0), (y1, v1, l1) = out
    assert l1 > l0
    assert np.array_equal(y0, y1) and np.array_equal(v0, v1)


def test_tc_bounded_wait_gives_nan_not_a_hang(ctx):
    """inject_timeout bit 2: the first CTA of the variance pass waits 5 ms on
    a barrier nothing signals and gives up; its points' s2 are NaN, the
    others and every yhat are finite, and the context keeps working."""
    g = np.random.default_rng(3)
    n, d, N = 300, 2, 300
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    model = ctx.fit(dev(x), dev(y), dev([3.0, 2.0]), 1.95, 1e-8, "fp64")
    xs = g.random((N, d))
    ctx.set_options(inject_timeout=2)
    try:
        yh, s2 = ctx.predict(model, dev(xs))
        yh, s2 = host(yh), host(s2)
    finally:
        ctx.set_options(inject_timeout=0)
    assert np.all(np.isfinite(yh))
    assert np.all(np.isnan(s2[:128])) and np.all(np.isfinite(s2[128:]))
    yh2, s22 = ctx.predict(model, dev(xs))
    assert np.all(np.isfinite(host(s22)))
    assert np.array_equal(host(yh2), yh)
    model.free()


def test_bench_kriging_only_runs():
    """bench.py --kriging-only (the entry the variance-pass profiles name)
    at a small size: one JSON line, positive times, no NaN variances."""
    import json
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--kriging-only", "--n", "300", "--points", "1000",
                        "--steps", "1", "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["unit"] == "points/s" and line["value"] > 0
    assert line["variance_nan"] == 0
    assert 0 < line["mean_only_s"] and 0 < line["mean_and_variance_s"]
    assert "tensor_core_pass_s" in line["variance_solve"]


def test_tc_workspace_beyond_budget_names_the_fp32_path():
    """A budget that holds the fit and the FP32-pipe prediction's scratch but
    not the tensor-core pass's slice tables: gp_predict with variances fails
    with GP_ENOMEM naming predict_tc, and succeeds with predict_tc = 0."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    n, d, N = 2048, 3, 500
    model_b = gp.call_bytes("fit", n, d)
    fit_ws = gp.call_bytes("nll_batch", n, d, 1, "fp64")
    tc_ws = gp.call_bytes("predict", n, d, N)
    budget = model_b + fit_ws + (4 << 20)
    assert tc_ws + model_b > budget
    g = np.random.default_rng(21)
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    c = gp.Context(0, hbm_budget_bytes=budget)
    try:
        model = c.fit(dev(x), dev(y), dev([2.0, 3.0, 4.0]), 1.95, 1e-8, "fp64")
        xs = dev(g.random((N, d)))
        with pytest.raises(gp.GPError) as e:
            c.predict(model, xs)
        assert e.value.code == gp.GP_ENOMEM and "predict_tc" in str(e.value)
        c.set_options(predict_tc=0)
        yh, s2 = c.predict(model, xs)
        assert torch.isfinite(s2).all() and torch.isfinite(yh).all()
        model.free()
    finally:
        c.close()


def test_tc_remainder_on_the_second_stream_gives_the_same_bits():
    """N = 2 x 152 x 128 + 300 points: two whole chunks (the second r slot)
    and a 3-block remainder whose pass runs on the context's second stream.
    The same bits as a budget that allows one block per chunk (no remainder
    path), every variance finite, sampled points against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    g = np.random.default_rng(31)
    n, d, N = 300, 3, 2 * 152 * 128 + 300
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    theta = np.array([2.0, 4.0, 3.0])
    xs = g.random((N, d))
    out = []
    for budget in (0, 6 << 20):
        c = gp.Context(0, hbm_budget_bytes=budget)
        try:
            model = c.fit(dev(x), dev(y), dev(theta), 1.95, 1e-8, "fp64")
            yh, s2 = c.predict(model, dev(xs))
            out.append((host(yh), host(s2)))
            model.free()
        finally:
            c.close()
    (y0, v0), (y1, v1) = out
    assert np.all(np.isfinite(v0))
    assert np.array_equal(y0, y1) and np.array_equal(v0, v1)
    idx = np.unique(np.r_[0, N - 1, np.arange(2 * 152 * 128 - 5, 2 * 152 * 128 + 5), g.integers(0, N, 100)])
    yo, so, _ = oracle.predict(x, y, theta, 1.95, 1e-8, xs[idx])
    o, _ = oracle.nll(x, y, theta, 1.95, 1e-8)
    assert np.max(np.abs(y0[idx] - yo)) <= 1e-8 * max(1.0, np.max(np.abs(yo)))
    assert np.max(np.abs(v0[idx] - so)) <= 1e-8 * o["sigma2"]
