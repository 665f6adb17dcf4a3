"""Condition estimate, the FP32-grade factorisation and GP_AUTO routing
(gp_nll_batch_ex) against the oracle and a closed form."""
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


def test_cond_estimate_kms_closed_form(ctx):
    """d = 1, x_i = i h, p = 1, delta = 0: R_ij = rho^|i-j| (Kac-Murdock-Szego).
    R^-1 is tridiagonal with column sums 1/(1-rho) at the ends and
    (1+rho)/(1-rho) inside, so ||R^-1||_1 = (1+rho)/(1-rho); ||R||_1 is the
    middle column's sum 1 + rho^a + rho^b + ... (geometric on both sides)."""
    for n, theta in ((300, 40.0), (517, 200.0)):
        h = 1.0 / n
        x = (np.arange(n) * h)[:, None]
        y = np.sin(7 * x[:, 0])
        rho = np.exp(-theta * h)
        inv1 = (1 + rho) / (1 - rho)
        cols = [sum(rho ** abs(i - j) for i in range(n)) for j in (n // 2, (n - 1) // 2)]
        exact = max(cols) * inv1
        res = ctx.nll_batch(dev(x), dev(y), dev([[theta]]), 1.0, 0.0, "mixed", cond=True)
        est = float(host(res["cond"])[0])
        print(f"\nKMS n={n} rho={rho:.4f}: cond1 exact {exact:.6e}, estimate {est:.6e}")
        # Hager's iteration reaches the exact norm here (the oracle's, in double,
        # to 1e-13); the split factor's error is cond 2^-40 ~ 2e-10
        assert abs(est / exact - 1) <= 1e-8


def spread_case():
    """n = 400, d = 3, delta = 1e-8, theta spread so that cond_1(R) runs from
    3e2 to 9e8 (from the oracle)."""
    g = np.random.default_rng(92)
    n, d, p, delta = 400, 3, 1.95, 1e-8
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = np.concatenate([inputs.log_uniform_thetas(g, 20, d, lo=-1.5, hi=2.0),
                         inputs.log_uniform_thetas(g, 6, d, lo=1.8, hi=2.5)])
    return x, y, th, p, delta


def test_cond_estimate_against_oracle(ctx):
    """The same iteration as the oracle's estimator: identical where the
    factor's error cannot change its decisions, a valid estimate elsewhere."""
    x, y, th, p, delta = spread_case()
    ref, st = oracle.nll_batch(x, y, th, p, delta, want_cond=True)
    res = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "mixed", cond=True)
    ok = (st == 0) & (host(res["status"]) == 0)
    c_or, c_gp = ref[ok, 6], host(res["cond"])[ok]
    ratio = c_gp / c_or
    well = c_or <= 1e6
    print(f"\ncond: {ok.sum()} candidates, {well.sum()} with cond <= 1e6; "
          f"max |ratio - 1| there {np.max(np.abs(ratio[well] - 1)):.2e}; ratio range {ratio.min():.3f}..{ratio.max():.3f}")
    assert well.sum() >= 5
    assert np.all(np.abs(ratio[well] - 1) <= 1e-5)
    assert np.all((ratio >= 0.2) & (ratio <= 5.0))
    # the estimate changes nothing else
    plain = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "mixed")
    for k in ("nll", "mu", "sigma2", "logdet", "status"):
        assert np.array_equal(host(plain[k]), host(res[k]), equal_nan=True)


def test_cond_needs_split_precision(ctx):
    from paper_1203_1269_gb300 import gp
    w = inputs.small_grid_fit()
    with pytest.raises(gp.GPError) as e:
        ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas[:2]), w.p, w.delta, "fp64", cond=True)
    assert e.value.code == gp.GP_ENOTSUP


def test_fp32_grade_within_its_bound(ctx):
    """GP_FP32 is the split factorisation with 3 slices: the same numbers as
    GP_MIXED at slices = 3, and within cond_1(R) 2^-30 of the oracle."""
    g = np.random.default_rng(91)
    n, d, p, delta = 500, 3, 1.95, 1e-3
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, 8, d, lo=1.0, hi=2.0)    # cond_1 4e3 .. 8e4
    ref, st = oracle.nll_batch(x, y, th, p, delta, want_cond=True)
    assert np.all(st == 0)
    r32 = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "fp32")
    try:
        ctx.set_options(slices=3)
        r3 = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "mixed")
    finally:
        ctx.set_options(slices=5)
    assert np.array_equal(host(r32["nll"]), host(r3["nll"]))
    rel = np.abs(host(r32["nll"]) - ref[:, 0]) / np.abs(ref[:, 0])
    bound = ref[:, 6] * 2.0 ** -30
    print(f"\nfp32-grade: max rel {rel.max():.2e}, max rel / bound {np.max(rel / bound):.2e}")
    assert np.all(rel <= bound)


@pytest.mark.parametrize("tol", [1e-6, 1e-3])
def test_auto_meets_tolerance(ctx, tol):
    """GP_AUTO: every candidate within auto_tol of the oracle, each from the
    cheapest arithmetic whose bound allowed it."""
    from paper_1203_1269_gb300 import gp
    x, y, th, p, delta = spread_case()
    ref, st = oracle.nll_batch(x, y, th, p, delta, want_cond=True)
    try:
        ctx.set_options(auto_tol=tol)
        res = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "auto", cond=True)
    finally:
        ctx.set_options(auto_tol=1e-6)
    used = host(res["prec_used"])
    sts = host(res["status"])
    assert np.array_equal(sts, st)
    ok = st == 0
    rel = np.abs(host(res["nll"])[ok] - ref[ok, 0]) / np.abs(ref[ok, 0])
    counts = {gp.PRECISION_NAMES[v]: int((used == v).sum()) for v in np.unique(used)}
    print(f"\nauto tol={tol:g}: routes {counts}, max rel err {rel.max():.2e}, cond {ref[ok, 6].min():.1e}..{ref[ok, 6].max():.1e}")
    assert np.all(rel <= tol)
    assert len(counts) == (3 if tol < 1e-5 else 2)
    # the routing follows the documented bounds on the reported estimates
    c = host(res["cond"])
    f32 = used == gp.GP_FP32
    assert np.all(c[f32] * 2.0 ** -30 <= tol)
    mix = used == gp.GP_MIXED
    assert np.all(c[mix] * 2.0 ** -46 <= tol)


def test_prec_used_reports_fixed_precision(ctx):
    from paper_1203_1269_gb300 import gp
    w = inputs.small_grid_fit()
    for name in ("fp64", "mixed", "fp32"):
        out = dict(prec_used=torch.full((8,), -9, dtype=torch.int32, device="cuda"))
        kw = dict(dtype=torch.float64, device="cuda")
        out.update(nll=torch.empty(8, **kw), mu=torch.empty(8, **kw), sigma2=torch.empty(8, **kw),
                   logdet=torch.empty(8, **kw), status=torch.empty(8, dtype=torch.int32, device="cuda"))
        ctx.nll_batch(dev(w.x), dev(w.y), dev(w.thetas[:8]), w.p, w.delta, name, out=out)
        assert np.all(host(out["prec_used"]) == gp.PRECISIONS[name])


def test_auto_chunked_matches_one_chunk(ctx):
    """GP_AUTO over a batch split into chunks of 5 (max_batch): every
    candidate's estimate, route and values are the same bits as in one chunk."""
    x, y, th, p, delta = spread_case()
    base = ctx.options()
    try:
        one = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "auto", cond=True)
        ctx.set_options(max_batch=5)
        many = ctx.nll_batch(dev(x), dev(y), dev(th), p, delta, "auto", cond=True)
    finally:
        ctx.set_options(**base)
    for k in ("nll", "mu", "sigma2", "logdet", "status", "cond", "prec_used"):
        assert np.array_equal(host(many[k]), host(one[k]), equal_nan=True), k
