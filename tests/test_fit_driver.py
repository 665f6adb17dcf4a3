"""The end-to-end fit driver (genetic search + double refinement + fit +
SSPE).  CPU: the search logic on a stand-in objective.  GPU: a small fit
whose final -2logL and SSPE match the oracle at the chosen theta."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1203_1269_gb300 import fit


class _Bowl:
    """Stand-in for gp.Context.nll_batch: a smooth bowl in log10 theta."""
    target = np.array([-0.7, 0.4])

    def nll_batch(self, x, y, th, p, delta, prec="mixed", out=None):
        z = np.log10(th.cpu().numpy())
        f = np.sum((z - self.target) ** 2, axis=1)
        return {"nll": torch.as_tensor(f), "status": torch.zeros(len(f), dtype=torch.int32)}


class _BowlGrad(_Bowl):
    """The same bowl with its gradient in theta, as gp.Context.nll_grad_batch
    returns it: d/dtheta_k sum (log10 theta - t)^2 = 2 (z_k - t_k) / (theta_k ln 10)."""

    def nll_grad_batch(self, x, y, th, p, delta):
        t = th.cpu().numpy()
        z = np.log10(t)
        f = np.sum((z - self.target) ** 2, axis=1)
        g = 2.0 * (z - self.target) / (t * np.log(10.0))
        return {"nll": torch.as_tensor(f), "grad": torch.as_tensor(g),
                "status": torch.zeros(len(f), dtype=torch.int32)}


class _Ridge(_BowlGrad):
    """A minimum outside the box in one coordinate: the search must stop on
    the boundary there (projected gradient)."""
    target = np.array([-0.7, 1.6])


def test_gradient_search_on_a_bowl():
    x = torch.zeros((5, 2), dtype=torch.float64)
    y = torch.zeros(5, dtype=torch.float64)
    z, f, evals, hist = fit.gradient_search(_BowlGrad(), x, y, 2.0, 0.0, starts=8, iterations=40, seed=5)
    assert all(a >= b for a, b in zip(hist, hist[1:]))
    assert f < 1e-10 and np.max(np.abs(z - _BowlGrad.target)) < 1e-5
    assert evals <= 8 * 41
    z2, f2, _, _ = fit.gradient_search(_BowlGrad(), x, y, 2.0, 0.0, starts=8, iterations=40, seed=5)
    assert np.array_equal(z2, z) and f2 == f                     # seeded: reproducible
    z4, f4, e4, _ = fit.gradient_search(_BowlGrad(), x, y, 2.0, 0.0, iterations=30, z0=np.array([[0.5, -1.5]]))
    assert e4 <= 31 and f4 < 1e-10                               # one given start
    zr, fr, _, _ = fit.gradient_search(_Ridge(), x, y, 2.0, 0.0, starts=8, iterations=60, seed=6)
    assert abs(zr[0] + 0.7) < 1e-4 and zr[1] == fit.HI            # on the box's edge
    assert abs(fr - 0.6 ** 2) < 1e-8


def test_genetic_search_and_refinement_on_a_bowl():
    ctx = _Bowl()
    x = torch.zeros((5, 2), dtype=torch.float64)
    y = torch.zeros(5, dtype=torch.float64)
    z, f, evals, hist = fit.genetic_search(ctx, x, y, 2.0, 0.0, generations=20, population=100, seed=3)
    assert evals == 2000
    assert all(a >= b for a, b in zip(hist, hist[1:]))          # best never gets worse
    assert f < 1e-3 and np.max(np.abs(z - _Bowl.target)) < 0.05
    z2, f2, used = fit.refine_double(ctx, x, y, 2.0, 0.0, z, f, evaluations=16)
    assert used <= 16 and f2 <= f
    z3, f3, _, _ = fit.genetic_search(ctx, x, y, 2.0, 0.0, generations=20, population=100, seed=3)
    assert np.array_equal(z3, z) and f3 == f                     # seeded: reproducible


@pytest.mark.gpu
def test_fit_driver_matches_oracle_at_chosen_theta():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1203_1269_gb300 import gp, inputs
    ctx = gp.Context(0)
    g = inputs.rng(77)
    x = inputs.random_lhd(g, 200, 2)
    y = inputs.y_trig2(x)
    xs = inputs.uniform_design(g, 300, 2)
    ys = inputs.y_trig2(xs)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    res = fit.fit_and_predict(ctx, dev(x), dev(y), 2.0, 1e-8, dev(xs), ys, generations=6, population=50,
                              refine_method="compass")
    res2 = fit.fit_and_predict(ctx, dev(x), dev(y), 2.0, 1e-8, dev(xs), ys, generations=6, population=50,
                               refine_method="compass")
    assert res["log10_theta"] == res2["log10_theta"] and res["nll"] == res2["nll"]
    th = 10.0 ** np.array(res["log10_theta"])
    o, st = oracle.nll(x, y, th, 2.0, 1e-8)
    assert st == 0
    assert abs(res["nll"] - o["nll"]) <= 1e-9 * abs(o["nll"]) + 1e-9
    assert res["nll"] <= res["nll_ga"] + 1e-6 * abs(res["nll_ga"])
    yo, _, _ = oracle.predict(x, y, th, 2.0, 1e-8, xs, want_var=False)
    sspe_o = float(np.sum((ys - yo) ** 2))
    assert abs(res["sspe"] - sspe_o) <= 1e-8 * max(1.0, sspe_o)
    ctx.close()


@pytest.mark.gpu
def test_gradient_search_reaches_the_genetic_optimum():
    """Multi-start gradient search on gp_nll_grad_batch: its optimum is no
    worse than the GA's (double-refined) one, and -2logL there is the
    oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1203_1269_gb300 import gp, inputs
    ctx = gp.Context(0)
    g = inputs.rng(78)
    x = inputs.random_lhd(g, 200, 2)
    y = inputs.y_trig2(x)
    xs = inputs.uniform_design(g, 300, 2)
    ys = inputs.y_trig2(xs)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    ga = fit.fit_and_predict(ctx, dev(x), dev(y), 2.0, 1e-8, dev(xs), ys, generations=10, population=60,
                             refine_method="compass")
    gr = fit.fit_and_predict(ctx, dev(x), dev(y), 2.0, 1e-8, dev(xs), ys, search="grad", starts=12, iterations=40)
    print(f"\nGA + refine: {ga['nll']:.6f} at {ga['log10_theta']} ({ga['evaluations']} evaluations); "
          f"gradient: {gr['nll']:.6f} at {gr['log10_theta']} ({gr['evaluations']} evaluations)")
    assert gr["nll"] <= ga["nll"] + 1e-6 * abs(ga["nll"])
    # the GA's best point refined by gradient steps instead of the compass search
    gg = fit.fit_and_predict(ctx, dev(x), dev(y), 2.0, 1e-8, dev(xs), ys, generations=10, population=60,
                             refine_method="grad")
    assert gg["nll"] <= ga["nll"] + 1e-9 * abs(ga["nll"])
    th = 10.0 ** np.array(gr["log10_theta"])
    o, st = oracle.nll(x, y, th, 2.0, 1e-8)
    assert st == 0 and abs(gr["nll"] - o["nll"]) <= 1e-9 * abs(o["nll"]) + 1e-9
    ctx.close()


def test_replicate_table_shapes_and_means(monkeypatch):
    """The replication harness runs one fit per replication with a fresh
    design and averages the five reported quantities per size."""
    calls = []

    def fake_fit(ctx, x, y, p, delta, xs, ys, prec="mixed", seed=0, **kw):
        calls.append((x.shape[0], x.shape[1], seed, float(x[0, 0])))
        n = x.shape[0]
        return {"seconds": 1.0 + seed, "nll": -n, "mu": 0.5, "sigma2": 2.0, "sspe": 3.0 * seed}

    monkeypatch.setattr(fit, "fit_and_predict", fake_fit)
    monkeypatch.setitem(fit.TABLES, "tiny", {"d": 2, "sizes": [(16, 3), (32, 2)], "y": "y_trig2"})
    rows = fit.replicate(None, "tiny", device=torch.device("cpu"))
    assert [r["n"] for r in rows] == [16, 32] and [r["replications"] for r in rows] == [3, 2]
    assert [c[:3] for c in calls] == [(16, 2, 0), (16, 2, 1), (16, 2, 2), (32, 2, 0), (32, 2, 1)]
    assert len({c[3] for c in calls[:3]}) == 3                     # a fresh design per replication
    assert rows[0]["seconds"] == 2.0 and rows[0]["nll"] == -16 and rows[0]["sspe"] == 3.0
    assert rows[1]["seconds"] == 1.5 and rows[1]["sspe"] == 1.5
    assert fit.TABLES["example1"]["sizes"][-1] == (512, 10) and fit.TABLES["example2"]["sizes"][-1] == (4064, 1)

