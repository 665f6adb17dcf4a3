"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 path): -2logL within 1e-9 relative and predictions within
1e-8 where the oracle's condition estimate of R is at most 1e8.  Beyond that
the two double-precision factorisations may legitimately differ by about
n * cond(R) * u in log|R| and the check is that bound (see cond_bound).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1203_1269_gb300 import inputs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def nll_tol(cond, n, tol=1e-9):
    """Relative tolerance on -2logL: `tol` where cond <= 1e8, else the
    rounding bound c * n * cond * u on the absolute error of log|R| and
    n log Q, divided by |-2logL| by the caller."""
    return tol if cond <= 1e8 else None


def compare_batch(w, res, ref, st_ref, tol=1e-9, label=""):
    nll = host(res["nll"]); mu = host(res["mu"]); s2 = host(res["sigma2"])
    ld = host(res["logdet"]); st = host(res["status"])
    worst = 0.0
    for t in range(len(st_ref)):
        assert st[t] == st_ref[t], (label, t, st[t], st_ref[t])
        if st_ref[t] != 0:
            continue
        cond = ref[t, 6]
        rel = abs(nll[t] - ref[t, 0]) / abs(ref[t, 0])
        if cond <= 1e8:
            assert rel <= tol, (label, t, rel, cond)
            assert abs(mu[t] - ref[t, 1]) <= 1e-8 * max(1.0, abs(ref[t, 1])), (label, t)
            assert abs(s2[t] - ref[t, 2]) <= 1e-8 * abs(ref[t, 2]), (label, t)
            assert abs(ld[t] - ref[t, 3]) <= tol * max(1.0, abs(ref[t, 0])), (label, t)
            worst = max(worst, rel)
        else:
            # both sides are backward-stable double factorisations: their
            # log|R| and n log Q differ by at most ~ c n cond u
            bound = 64.0 * w.n * cond * U * (1.0 + w.n)
            assert abs(nll[t] - ref[t, 0]) <= max(bound, tol * abs(ref[t, 0])), (label, t, cond)
    return worst


def test_assemble_dense_matches_oracle(ctx):
    g = np.random.default_rng(1)
    for (n, d, p, delta) in [(1, 1, 2.0, 0.0), (37, 3, 1.95, 1e-6), (300, 5, 1.5, 0.0), (129, 2, 2.0, 1e-8)]:
        x = g.random((n, d))
        th = 10 ** g.uniform(-2, 1, d)
        R = host(ctx.corr_assemble(dev(x), dev(th), p, delta, "dense"))
        Ro = oracle.corr_matrix(x, th, p, delta)
        assert np.max(np.abs(R - Ro) / np.maximum(np.abs(Ro), 1e-300)) < 1e-14
        assert np.array_equal(R, R.T)


def unpack_tiles(buf, n, nb=128):
    nt = (n + nb - 1) // nb
    full = np.zeros((nt * nb, nt * nb))
    idx = 0
    for J in range(nt):
        for I in range(J, nt):
            tile = buf[idx * nb * nb:(idx + 1) * nb * nb].reshape(nb, nb).T  # column-major
            full[I * nb:(I + 1) * nb, J * nb:(J + 1) * nb] = tile
            idx += 1
    return full


@pytest.mark.parametrize("n", [1, 5, 127, 128, 129, 300])
def test_assemble_tiles_layout(ctx, n):
    g = np.random.default_rng(n)
    d, p, delta = 4, 1.95, 1e-7
    x = g.random((n, d))
    th = 10 ** g.uniform(-2, 1, d)
    buf = host(ctx.corr_assemble(dev(x), dev(th), p, delta, "tiles"))
    full = unpack_tiles(buf, n)
    Ro = oracle.corr_matrix(x, th, p, delta)
    low = np.tril(full[:n, :n])
    assert np.max(np.abs(low - np.tril(Ro))) < 1e-14
    npad = full.shape[0]
    # padding: identity on the diagonal, zeros elsewhere (lower tiles)
    pad = np.tril(full)[n:, :]
    expect = np.zeros_like(pad)
    for i in range(n, npad):
        expect[i - n, i] = 1.0
    assert np.array_equal(pad, expect)


def test_nll_batch_small_grid(ctx):
    """Every candidate of the n=200, d=2 theta grid against the oracle."""
    w = inputs.small_grid_fit()
    ref, st = oracle.nll_batch(w.x, w.y, w.thetas, w.p, w.delta, want_cond=True)
    res = ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas), w.p, w.delta, "fp64")
    worst = compare_batch(w, res, ref, st, label="grid64")
    print(f"\nn=200 grid: worst rel err (cond<=1e8) {worst:.3e}; "
          f"cond range {ref[:, 6].min():.2e}..{ref[:, 6].max():.2e}")


@pytest.mark.parametrize("n", [2, 3, 64, 127, 128, 129, 255, 256, 257, 389])
def test_nll_batch_ragged_sizes(ctx, n):
    g = np.random.default_rng(100 + n)
    d, p, delta = 3, 1.95, 1e-6
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, 12, d, lo=-1.0, hi=1.0)
    ref, st = oracle.nll_batch(x, y, th, p, delta, want_cond=True)
    res = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "fp64")
    compare_batch(type("W", (), {"n": n})(), res, ref, st, label=f"n{n}")


def test_status_cases(ctx):
    # n = 1: Q = 0 -> degenerate, -inf
    res = ctx.nll_batch(dev([[0.3, 0.7]]), dev([2.5]), dev([[1.0, 2.0]]), 1.9, 1e-3, "fp64")
    assert host(res["status"])[0] == -6 and host(res["nll"])[0] == -math.inf
    assert abs(host(res["logdet"])[0] - math.log(1.001)) < 1e-12
    # duplicate points with delta = 0 -> not positive definite; negative theta -> EINVAL
    x = np.array([[0.2, 0.3], [0.2, 0.3], [0.7, 0.1], [0.5, 0.9]])
    y = np.array([1.0, 2.0, 0.5, -1.0])
    th = np.array([[1.0, 1.0], [-1.0, 1.0], [1.0, float("nan")], [2.0, 3.0]])
    res = ctx.nll_batch(dev(x), dev(y), dev(th), 2.0, 0.0, "fp64")
    st = host(res["status"])
    assert list(st) == [-3, -1, -1, -3]
    assert host(res["nll"])[0] == math.inf
    # the same with a nugget: fine, and equal to the oracle
    res = ctx.nll_batch(dev(x), dev(y), dev(th[[0, 3]]), 2.0, 1e-6, "fp64")
    for t, row in enumerate(th[[0, 3]]):
        o, s = oracle.nll(x, y, row, 2.0, 1e-6)
        assert s == 0 and host(res["status"])[t] == 0
        assert abs(host(res["nll"])[t] - o["nll"]) <= 1e-9 * abs(o["nll"])


def test_bad_arguments_rejected(ctx):
    from paper_1203_1269_gb300 import gp
    x = dev(np.random.rand(4, 2)); y = dev(np.random.rand(4)); th = dev([[1.0, 1.0]])
    for p in (0.0, 2.5, float("nan")):
        with pytest.raises(gp.GPError):
            ctx.nll_batch(x, y, th, p, 0.0)
    with pytest.raises(gp.GPError):
        ctx.nll_batch(x, y, th, 2.0, -1.0)


def kms_closed_form(n, rho, y):
    c = 1.0 / (1.0 - rho * rho)
    one = np.ones(n)

    def qf(u, v):
        diag = np.full(n, 1.0 + rho * rho)
        diag[0] = diag[-1] = 1.0
        return c * (np.dot(u * diag, v) - rho * (np.dot(u[1:], v[:-1]) + np.dot(u[:-1], v[1:])))
    A, B, C = qf(one, one), qf(one, y), qf(y, y)
    mu = B / A
    Q = C - B * B / A
    logdet = (n - 1) * math.log(1.0 - rho * rho)
    return logdet + n * math.log(Q), mu, Q / n, logdet


@pytest.mark.parametrize("n", [1000, 4000])
def test_kms_closed_form_large(ctx, n):
    """d = 1, x_i = i/1024, p = 1, delta = 0: R_ij = rho^|i-j| (Kac-Murdock-
    Szego); log|R|, mu_hat, sigma2_hat and -2logL in closed form at any n."""
    h = 1.0 / 1024.0
    x = (np.arange(n) * h).reshape(n, 1)
    g = np.random.default_rng(7)
    y = g.standard_normal(n)
    rhos = [0.3, 0.8, 0.95]
    th = np.array([[-math.log(r) / h] for r in rhos])
    res = ctx.nll_batch(dev(x), dev(y), dev(th), 1.0, 0.0, "fp64")
    for t, r in enumerate(rhos):
        rho = math.exp(-th[t, 0] * h)
        nll, mu, s2, ld = kms_closed_form(n, rho, y)
        assert host(res["status"])[t] == 0
        assert abs(host(res["nll"])[t] - nll) <= 1e-9 * abs(nll)
        assert abs(host(res["logdet"])[t] - ld) <= 1e-9 * abs(ld)
        assert abs(host(res["mu"])[t] - mu) <= 1e-8 * max(1, abs(mu))
        assert abs(host(res["sigma2"])[t] - s2) <= 1e-8 * s2


def test_batch_results_independent_of_batch(ctx):
    """Each candidate's result is bit-identical alone and inside a batch."""
    w = inputs.small_grid_fit(n=300, N=0)
    res = ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas), w.p, w.delta, "fp64")
    for t in (0, 17, 63):
        one = ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas[t:t + 1]), w.p, w.delta, "fp64")
        for k in ("nll", "mu", "sigma2", "logdet"):
            assert host(one[k])[0] == host(res[k])[t]


def test_host_entry_point_matches_device(ctx):
    w = inputs.small_grid_fit(n=150, N=0)
    res = ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas[:8]), w.p, w.delta, "fp64")
    hres = ctx.nll_batch_host(torch.from_numpy(w.x.copy()), torch.from_numpy(w.y.copy()),
                              torch.from_numpy(w.thetas[:8].copy()), w.p, w.delta, "fp64")
    for k in ("nll", "mu", "sigma2", "logdet", "status"):
        assert np.array_equal(host(res[k]), hres[k].numpy())


def test_fit_predict_matches_oracle(ctx):
    w = inputs.small_grid_fit()
    theta = np.array([3.0, 5.0])
    model = ctx.fit(dev(w.x), dev(w.y), dev(theta), w.p, w.delta, "fp64")
    o, st = oracle.nll(w.x, w.y, theta, w.p, w.delta, want_cond=True)
    assert st == 0
    assert abs(model.nll - o["nll"]) <= 1e-9 * abs(o["nll"])
    yh, s2 = ctx.predict(model, dev(w.xs))
    yo, so, st = oracle.predict(w.x, w.y, theta, w.p, w.delta, w.xs)
    yh, s2 = host(yh), host(s2)
    scale_y = np.max(np.abs(yo))
    assert np.max(np.abs(yh - yo)) <= 1e-8 * scale_y
    assert np.max(np.abs(s2 - so)) <= 1e-8 * o["sigma2"]
    # mean only
    yh2, none = ctx.predict(model, dev(w.xs), want_var=False)
    assert none is None and np.array_equal(host(yh2), yh)
    model.free()


def test_predict_in_many_launches():
    """N = 20000 test points take several launches (at most four waves of
    CTAs each), and a budget that leaves room for few CTAs' scratch takes
    many more: the predictions are the same bits either way, and sampled
    points (both ends, the launch boundaries) match the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    g = np.random.default_rng(81)
    n, d, N = 200, 3, 20000
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    theta = np.array([2.0, 4.0, 3.0])
    xs = g.random((N, d))
    out = {}
    for budget in (0, 2 << 20):
        c = gp.Context(0, hbm_budget_bytes=budget)
        try:
            model = c.fit(dev(x), dev(y), dev(theta), 1.95, 1e-8, "fp64")
            before = c.launch_count()
            yh, s2 = c.predict(model, dev(xs))
            out[budget] = (host(yh), host(s2), c.launch_count() - before)
            model.free()
        finally:
            c.close()
    (y0, v0, l0), (y1, v1, l1) = out[0], out[2 << 20]
    assert l0 >= 2 and l1 > l0
    assert np.array_equal(y0, y1) and np.array_equal(v0, v1)
    idx = np.unique(np.r_[0, 1, N - 1, np.arange(9700, 9760), np.arange(19440, 19470),
                          g.integers(0, N, 200)])
    yo, so, st = oracle.predict(x, y, theta, 1.95, 1e-8, xs[idx])
    o, _ = oracle.nll(x, y, theta, 1.95, 1e-8, want_cond=True)
    assert np.max(np.abs(y0[idx] - yo)) <= 1e-8 * max(1.0, np.max(np.abs(yo)))
    assert np.max(np.abs(v0[idx] - so)) <= 1e-8 * o["sigma2"]


@pytest.mark.parametrize("d", [17, 64])
def test_wide_designs_up_to_max_d(ctx, d):
    """d just past the assembly kernels' register-bounded variants (17) and
    the largest d the library accepts (64): -2logL at both precisions and
    kriging against the oracle; d = 65 is rejected."""
    from paper_1203_1269_gb300 import gp
    g = np.random.default_rng(90 + d)
    n, T, p, delta = 300, 4, 1.95, 1e-6
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, T, d, lo=-1.5, hi=-0.5)
    ref, st = oracle.nll_batch(x, y, th, p, delta, want_cond=True)
    assert np.all(st == 0) and np.all(ref[:, 6] <= 1e8)
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-6)):
        res = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, prec)
        assert np.all(host(res["status"]) == 0)
        rel = np.abs(host(res["nll"]) - ref[:, 0]) / np.abs(ref[:, 0])
        assert rel.max() <= tol, (prec, rel.max())
    model = ctx.fit(dev(x), dev(y), dev(th[0]), p, delta, "fp64")
    xs = g.random((50, d))
    yh, s2 = ctx.predict(model, dev(xs))
    yo, so, _ = oracle.predict(x, y, th[0], p, delta, xs)
    assert np.max(np.abs(host(yh) - yo)) <= 1e-8 * max(1.0, np.max(np.abs(yo)))
    assert np.max(np.abs(host(s2) - so)) <= 1e-8 * model.sigma2
    model.free()
    if d == 64:
        x65 = g.random((n, 65))
        with pytest.raises(gp.GPError) as e:
            ctx.nll_batch(dev(x65), dev(y), dev(g.random((1, 65))), p, delta, "fp64")
        assert e.value.code == gp.GP_EINVAL


@pytest.mark.parametrize("n", [1, 129, 260])
def test_fit_predict_ragged_and_interpolation(ctx, n):
    g = np.random.default_rng(n + 5)
    d = 3
    x = g.random((n, d))
    y = np.cos(3 * x).sum(axis=1)
    theta = np.array([4.0, 2.0, 6.0])
    p = 1.95
    delta = 0.0 if n > 1 else 1e-6
    model = ctx.fit(dev(x), dev(y), dev(theta), p, delta, "fp64")
    xs = np.vstack([x[: min(n, 40)], g.random((37, d))])
    yh, s2 = ctx.predict(model, dev(xs))
    yo, so, st = oracle.predict(x, y, theta, p, delta, xs)
    yh, s2 = host(yh), host(s2)
    sig = max(model.sigma2, 1e-300)
    if n > 1:
        assert np.max(np.abs(yh - yo)) <= 1e-8 * max(1, np.max(np.abs(yo)))
        assert np.max(np.abs(s2 - so)) <= 1e-8 * sig + 1e-12
        # interpolation at the design points when delta = 0
        k = min(n, 40)
        assert np.max(np.abs(yh[:k] - y[:k])) <= 1e-6
    model.free()


def test_full_size_sampled_against_oracle(ctx):
    """n = 4000, d = 6, T = 256 (the benchmark's launch): every output is
    finite with a valid status, and a sample of candidates matches the oracle
    evaluated one by one."""
    w = inputs.hartman_shape()
    res = ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas), w.p, w.delta, "fp64")
    st = host(res["status"])
    assert np.all(st == 0)
    assert np.all(np.isfinite(host(res["nll"])))
    sample = np.linspace(0, w.T - 1, 16).astype(int)
    ref, st_ref = oracle.nll_batch(w.x, w.y, w.thetas[sample], w.p, w.delta, want_cond=True)
    sub = {k: v[torch.as_tensor(sample, device="cuda")] for k, v in res.items()}
    worst = compare_batch(w, sub, ref, st_ref, label="n4000")
    print(f"\nn=4000 sample: worst rel err (cond<=1e8) {worst:.3e}; cond "
          f"{ref[:, 6].min():.2e}..{ref[:, 6].max():.2e}")


def test_model_outlives_context_and_clean_exit():
    """A model freed after its context, and a process that exits holding a
    context and a model, both end cleanly."""
    import subprocess
    import sys
    from paper_1203_1269_gb300 import gp
    c2 = gp.Context(0)
    w = inputs.small_grid_fit(n=150, N=10)
    m = c2.fit(dev(w.x), dev(w.y), dev([3.0, 5.0]), w.p, w.delta, "fp64")
    c2.close()
    m.free()
    code = ("import numpy as np, torch\n"
            "from paper_1203_1269_gb300 import gp, inputs\n"
            "c = gp.Context(0)\n"
            "w = inputs.small_grid_fit(n=150, N=10)\n"
            "d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device='cuda')\n"
            "m = c.fit(d(w.x), d(w.y), d([3.0, 5.0]), w.p, w.delta, 'fp64')\n"
            "print('ok')\n")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "ok" in r.stdout


@pytest.mark.parametrize("p", [0.6, 1.95])
def test_assemble_tiles_power_across_scales(ctx, p):
    """The double assembly's table powers (|dx| = 2^m F_j (1 + u) for 2^-60 <=
    |dx| < 2^5, pow outside) against the oracle's pow, for coordinate
    differences from 2^-70 to 2^6 in one dimension (S up to about 50).  Each
    side rounds S to about an ulp, which exp(-S) turns into a relative error
    of S ulps, so the entries agree within 8 (1 + S) 2^-53 relative; a
    power wrong by a few ulps or more fails that."""
    g = np.random.default_rng(90)
    n = 300
    x = np.empty((n, 2))
    x[:, 0] = np.sort(2.0 ** g.uniform(-70.0, 6.0, n)) * np.where(g.random(n) < 0.5, -1.0, 1.0)
    x[:, 1] = g.random(n)
    th = np.array([30.0 / 64.0 ** p, 2.0])
    buf = host(ctx.corr_assemble(dev(x), dev(th), p, 1e-8, "tiles"))
    full = unpack_tiles(buf, n)
    Ro = oracle.corr_matrix(x, th, p, 1e-8)
    low, ref = np.tril(full[:n, :n]), np.tril(Ro)
    mask = ref > 0
    assert np.all(low[~mask] == 0.0)
    S = -np.log(ref[mask])
    rel = np.abs(low[mask] - ref[mask]) / ref[mask]
    assert np.all(rel <= 8.0 * 2.0 ** -53 * (1.0 + np.maximum(S, 0.0))), np.max(rel / (1.0 + np.abs(S)))
