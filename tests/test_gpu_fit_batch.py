"""gp_fit_batch (a batch of candidates, then the fit of the best one from its
own factor) and gp_fit in split precision: the model equals a fresh fit at
the best candidate, in double precision bit for bit, and the split model's
kriging means and variances stay within their stated error against the
oracle (means about cond 2^-46, variances about cond 2^-40)."""
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


def case(seed=811, n=600, d=4, T=12, N=200):
    g = np.random.default_rng(seed)
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, T, d, lo=-0.5, hi=1.0)
    xs = inputs.uniform_design(g, N, d)
    return x, y, th, 1.95, 1e-6, xs


def best_of(res):
    st, nll = host(res["status"]), host(res["nll"])
    ok = np.where(st == 0)[0]
    return int(ok[np.argmin(nll[ok])])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fit_batch_equals_fit_at_best(ctx, prec):
    x, y, th, p, delta, xs = case()
    X, Y, TH, XS = dev(x), dev(y), dev(th), dev(xs)
    out, best, model = ctx.fit_batch(X, Y, TH, p, delta, prec)
    ref = ctx.nll_batch(X, Y, TH, p, delta, prec)
    for k in ("nll", "mu", "sigma2", "logdet", "status"):
        assert torch.equal(out[k], ref[k]), k
    assert best == best_of(ref)
    fresh = ctx.fit(X, Y, TH[best].contiguous(), p, delta, prec)
    yh1, s1 = ctx.predict(model, XS)
    yh2, s2 = ctx.predict(fresh, XS)
    assert torch.equal(yh1, yh2) and torch.equal(s1, s2)
    assert (model.nll, model.mu, model.sigma2, model.logdet) == (fresh.nll, fresh.mu, fresh.sigma2, fresh.logdet)
    assert model.nll == float(host(ref["nll"])[best])
    model.free()
    fresh.free()


def test_fit_batch_refits_a_best_from_an_earlier_chunk(ctx):
    """With chunks of 4 candidates and the best one first, its factor is gone
    by the end of the batch: it is factored again, with the same result."""
    x, y, th, p, delta, xs = case(seed=812)
    X, Y, XS = dev(x), dev(y), dev(xs)
    ref = ctx.nll_batch(X, Y, dev(th), p, delta, "mixed")
    b = best_of(ref)
    order = [b] + [t for t in range(len(th)) if t != b]
    TH = dev(th[order])
    base = ctx.options()
    try:
        ctx.set_options(max_batch=4)
        out, best, model = ctx.fit_batch(X, Y, TH, p, delta, "mixed")
    finally:
        ctx.set_options(**base)
    assert best == 0
    fresh = ctx.fit(X, Y, TH[0].contiguous(), p, delta, "mixed")
    assert torch.equal(ctx.predict(model, XS)[1], ctx.predict(fresh, XS)[1])
    model.free()
    fresh.free()


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_split_fit_kriging_against_oracle(ctx, prec):
    x, y, th, p, delta, xs = case(seed=813)
    X, Y, TH, XS = dev(x), dev(y), dev(th), dev(xs)
    out, best, model = ctx.fit_batch(X, Y, TH, p, delta, prec)
    o, st = oracle.nll(x, y, th[best], p, delta, want_cond=True)
    assert st == 0
    cond = o["cond1"]
    yo, so, sto = oracle.predict(x, y, th[best], p, delta, xs)
    assert sto == 0
    yh, s2 = ctx.predict(model, XS)
    em = np.max(np.abs(host(yh) - yo)) / np.max(np.abs(y))
    ev = np.max(np.abs(host(s2) - so)) / o["sigma2"]
    # the split factor's unit: 2^-40 with 5 slices, 2^-30 with 3 (gp.h, GP_FP32)
    u = 2.0 ** -40 if prec == "mixed" else 2.0 ** -30
    print(f"\n{prec} fit at best of {len(th)} (cond1 {cond:.1e}): mean {em:.2e}, variance {ev:.2e} "
          f"(of sigma2); bounds {cond * u:.1e}, {16 * cond * u:.1e}")
    assert em <= cond * u
    assert ev <= 16 * cond * u
    # -2logL as gp_nll_batch gives it at this precision: within the split
    # factor's rounding bound n cond u
    assert abs(model.nll - o["nll"]) <= len(x) * cond * u
    model.free()


def test_concurrent_contexts_with_different_shapes():
    """Contexts on four threads fit, assemble and predict with different d at
    once.  Kernels whose shared memory depends on d raise their limit from
    several threads; the limit may only grow, so no launch is refused."""
    import threading
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    errors = []

    def work(d, seed):
        try:
            s = torch.cuda.Stream()
            c = gp.Context(0, stream=s)
            with torch.cuda.stream(s):
                g = np.random.default_rng(seed)
                x = inputs.random_lhd(g, 300, d)
                y = inputs.y_sinsum(x)
                th = inputs.log_uniform_thetas(g, 4, d, lo=-0.5, hi=0.5)
                xs = inputs.uniform_design(g, 500, d)
                X, Y, TH, XS = dev(x), dev(y), dev(th), dev(xs)
                for prec in ("fp64", "mixed"):
                    _, _, m = c.fit_batch(X, Y, TH, 1.95, 1e-6, prec)
                    for _ in range(10):
                        c.predict(m, XS)
                        c.nll_batch(X, Y, TH, 1.95, 1e-6, "mixed")
                    m.free()
                torch.cuda.synchronize()
            c.close()
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(d, 900 + d)) for d in (2, 5, 9, 12)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors


def test_fp64_lookahead_gives_the_same_bits(ctx):
    """Batches of up to 16 instances factor in double with a look-ahead (the
    next block column's diagonal step and panel on a second stream beside the
    rest of the update); larger ones without.  Every tile takes its updates in
    the same order, so 20 candidates in one batch and the same candidates one
    at a time (and in a batch of 3) give the same bits; gp_fit's model holds
    them too.  n = 700 (6 block columns, a ragged last one), p = 1.9."""
    g = np.random.default_rng(515)
    n, d = 700, 5
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, 20, d, lo=-1.0, hi=1.0)
    X, Y = dev(x), dev(y)
    big = ctx.nll_batch(X, Y, dev(th), 1.9, 1e-6, "fp64")
    three = ctx.nll_batch(X, Y, dev(th[:3]), 1.9, 1e-6, "fp64")
    for k in ("nll", "mu", "sigma2", "logdet", "status"):
        assert torch.equal(three[k], big[k][:3]), k
    for t in (0, 7, 19):
        one = ctx.nll_batch(X, Y, dev(th[t:t + 1]), 1.9, 1e-6, "fp64")
        for k in ("nll", "mu", "sigma2", "logdet"):
            assert torch.equal(one[k][0], big[k][t]), (t, k)
        model = ctx.fit(X, Y, dev(th[t]), 1.9, 1e-6, "fp64")
        assert model.nll == float(big["nll"][t])
        model.free()
