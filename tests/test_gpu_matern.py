"""The Matern correlation family (gp_options.correlation) against the oracle:
assembly in both storage layouts, -2logL in double and split precision, and
kriging from a fit (which keeps the family it was made with)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1203_1269_gb300 import inputs

pytestmark = pytest.mark.gpu

FAMS = ["matern12", "matern32", "matern52"]


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


def unpack_lower(buf, n, nb=128):
    nt = (n + nb - 1) // nb
    full = np.zeros((nt * nb, nt * nb))
    q = 0
    for J in range(nt):
        for I in range(J, nt):
            full[I * nb:(I + 1) * nb, J * nb:(J + 1) * nb] = buf[q * nb * nb:(q + 1) * nb * nb].reshape(nb, nb).T
            q += 1
    return full[:n, :n]


def case(seed, n=300, d=3, T=10, lo=-0.3, hi=1.3):
    g = np.random.default_rng(seed)
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, T, d, lo=lo, hi=hi)
    return x, y, th


class family:
    def __init__(self, ctx, fam):
        self.ctx, self.fam = ctx, fam

    def __enter__(self):
        self.ctx.set_options(correlation=self.fam)

    def __exit__(self, *a):
        self.ctx.set_options(correlation="powexp")


@pytest.mark.parametrize("fam", FAMS)
def test_matern_assembly(ctx, fam):
    x, _, th = case(51)
    n = x.shape[0]
    Ro = oracle.corr_matrix(x, th[0], 1.95, 1e-6, corr=fam)
    low = np.tril(Ro)
    m = low > 2.0 ** -120
    with family(ctx, fam):
        f64 = unpack_lower(host(ctx.corr_assemble(dev(x), dev(th[0]), 1.95, 1e-6, "tiles")), n)
        buf = host(ctx.corr_assemble(dev(x), dev(th[0]), 1.95, 1e-6, "tiles_df")).view(np.float32)
        dfv = unpack_lower(buf[0::2].astype(np.float64) + buf[1::2].astype(np.float64), n)
        dense = host(ctx.corr_assemble(dev(x), dev(th[0]), 1.95, 1e-6, "dense")).reshape(n, n)
    rel64 = np.abs(f64[m] - low[m]) / low[m]
    reldf = np.abs(dfv[m] - low[m]) / low[m]
    print(f"\n{fam}: FP64 tiles max rel {rel64.max():.2e}, double-float {reldf.max():.2e}")
    assert rel64.max() <= 1e-13
    # S = sum_k h_k as in the power-exponential case: the bound grows with S
    S = -np.log(np.maximum(low[m] - 1e-6 * (low[m] > 1.0), 2.0 ** -126))
    assert np.all(reldf <= 4e-14 + 1.5e-13 * S)
    assert np.max(np.abs(dense - Ro) / np.maximum(Ro, 2.0 ** -120)) <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("fam", FAMS)
def test_matern_nll(ctx, fam, prec):
    x, y, th = case(52, n=389, d=3, T=12)
    ref, st = oracle.nll_batch(x, y, th, 1.95, 1e-6, want_cond=True, corr=fam)
    with family(ctx, fam):
        res = ctx.nll_batch(dev(x), dev(y), dev(th), 1.95, 1e-6, prec)
    assert np.array_equal(host(res["status"]), st)
    ok = (st == 0) & (ref[:, 6] <= 1e8)
    rel = np.abs(host(res["nll"])[ok] - ref[ok, 0]) / np.abs(ref[ok, 0])
    tol = 1e-9 if prec == "fp64" else 1e-6
    print(f"\n{fam} {prec}: {ok.sum()} candidates with cond <= 1e8 (cond {ref[:, 6].min():.1e}..{ref[:, 6].max():.1e}), "
          f"max rel {rel.max():.2e}")
    assert ok.sum() >= 6 and rel.max() <= tol
    for k, col in (("mu", 1), ("sigma2", 2)):
        relk = np.abs(host(res[k])[ok] - ref[ok, col]) / np.maximum(np.abs(ref[ok, col]), 1e-300)
        assert relk.max() <= (1e-8 if prec == "fp64" else 1e-5)


def test_matern_half_equals_exponential(ctx):
    """nu = 1/2 is eq. (2) with p = 1 (up to rounding order)."""
    x, y, th = case(53, n=257, d=2, T=6)
    with family(ctx, "matern12"):
        a = host(ctx.nll_batch(dev(x), dev(y), dev(th), 1.3, 1e-6, "fp64")["nll"])
    b = host(ctx.nll_batch(dev(x), dev(y), dev(th), 1.0, 1e-6, "fp64")["nll"])
    assert np.max(np.abs(a - b) / np.abs(b)) <= 1e-12


@pytest.mark.parametrize("fam", ["matern32", "matern52"])
def test_matern_fit_predict(ctx, fam):
    x, y, th = case(54, n=260, d=3, T=1, lo=0.3, hi=0.9)
    g = np.random.default_rng(55)
    xs = np.vstack([x[:20], g.random((45, 3))])
    with family(ctx, fam):
        model = ctx.fit(dev(x), dev(y), dev(th[0]), 1.95, 1e-8, "fp64")
    # the fit keeps its family: predict with the context back on power-exponential
    yh, s2 = ctx.predict(model, dev(xs))
    o, st = oracle.nll(x, y, th[0], 1.95, 1e-8, corr=fam)
    yo, so, sto = oracle.predict(x, y, th[0], 1.95, 1e-8, xs, corr=fam)
    assert st == 0 and sto == 0
    assert abs(model.nll - o["nll"]) <= 1e-9 * abs(o["nll"])
    yh, s2 = host(yh), host(s2)
    print(f"\n{fam} kriging: max |dy| {np.max(np.abs(yh - yo)):.2e}, max |ds2| {np.max(np.abs(s2 - so)):.2e}")
    assert np.max(np.abs(yh - yo)) <= 1e-8 * max(1.0, np.max(np.abs(yo)))
    assert np.max(np.abs(s2 - so)) <= 1e-8 * model.sigma2 + 1e-12
    model.free()


def test_matern_ignores_p_and_rejects_bad_family(ctx):
    from paper_1203_1269_gb300 import gp
    x, y, th = case(56, n=130, d=2, T=2)
    with family(ctx, "matern52"):
        a = host(ctx.nll_batch(dev(x), dev(y), dev(th), 0.7, 0.0, "fp64")["nll"])
        b = host(ctx.nll_batch(dev(x), dev(y), dev(th), 5.0, 0.0, "fp64")["nll"])   # p out of (0, 2]: ignored
    assert np.array_equal(a, b)
    with pytest.raises(gp.GPError):
        ctx.set_options(correlation=7)
