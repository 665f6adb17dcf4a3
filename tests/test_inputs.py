"""CPU tests: the seeded input generators follow the stated recipe (shapes,
value ranges, Latin-hypercube structure, the serving stream's mix) and are
reproducible from their seeds."""
import numpy as np

from paper_1203_1269_gb300 import inputs


def test_random_lhd_is_latin():
    g = inputs.rng(5)
    for n, d in ((1, 1), (7, 3), (257, 6)):
        x = inputs.random_lhd(g, n, d)
        assert x.shape == (n, d) and np.all(x >= 0) and np.all(x < 1)
        for k in range(d):   # one point in each of the n strata of every axis
            assert np.array_equal(np.sort(np.floor(x[:, k] * n).astype(int)), np.arange(n))


def test_generators_are_seeded():
    a, b = inputs.hartman_shape(n=300, T=8), inputs.hartman_shape(n=300, T=8)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y) and np.array_equal(a.thetas, b.thetas)
    c = inputs.hartman_shape(n=300, T=8, seed=inputs.BASE_SEED + 99)
    assert not np.array_equal(a.x, c.x)


def test_theta_draws():
    g = inputs.rng(6)
    th = inputs.log_uniform_thetas(g, 4000, 3)
    assert th.shape == (4000, 3)
    assert th.min() >= 10.0 ** -2 and th.max() < 10.0
    # log10 theta uniform: its mean is the midpoint and a quarter falls in each quarter
    lt = np.log10(th)
    assert abs(lt.mean() + 0.5) < 0.05
    assert abs(np.mean(lt < -1.25) - 0.25) < 0.03
    grid = inputs.grid_thetas(2, 8)
    assert grid.shape == (64, 2) and len({tuple(r) for r in grid}) == 64
    assert np.isclose(grid.min(), 0.01) and np.isclose(grid.max(), 10.0)


def test_workload_recipes():
    w = inputs.small_grid_fit()
    assert (w.n, w.d, w.T, w.p, w.delta, w.xs.shape) == (200, 2, 64, 2.0, 1e-8, (1000, 2))
    w = inputs.hartman_shape()
    assert (w.n, w.d, w.T, w.p, w.delta) == (4000, 6, 256, 1.95, 1e-7)
    assert np.all(np.log10(w.thetas) >= -2) and np.all(np.log10(w.thetas) < 1)
    w = inputs.batched_split(n=256, T=16)
    assert (w.d, w.p, w.delta) == (8, 2.0, 1e-6)
    w = inputs.large_instance(n=512, N=100)
    assert (w.d, w.T, w.p, w.delta, w.xs.shape) == (10, 32, 1.9, 1e-6, (100, 10))


def test_responses_are_the_stated_functions():
    x = np.array([[0.25, 0.5, 0.75], [0.1, 0.2, 0.3]])
    s = np.sin(2 * np.pi * x)
    want = s[:, 0] + s[:, 1] / 2 + s[:, 2] / 3 + 0.1 * (x ** 2).sum(axis=1)
    assert np.allclose(inputs.y_sinsum(x), want, rtol=0, atol=1e-15)
    assert np.isclose(inputs.y_trig2(np.array([[0.25, 0.0]]))[0], 1.0 + 0.5)
    assert np.isclose(inputs.y_bump(np.array([[0.5, 0.5]]))[0], 1.0 + 0.05)


def test_serving_stream_mix():
    reqs = inputs.serving_stream(count=2000)
    assert reqs[0].kind == "fit"
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(reqs) / t[-1] - 200.0) < 20.0          # Poisson at 200/s
    kinds = np.array([r.kind == "fit" for r in reqs])
    assert abs(kinds.mean() - 0.5) < 0.05
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 256 and ns.max() <= 8192
    # log-uniform n: the median is near the geometric midpoint sqrt(256 * 8192)
    assert abs(np.log(np.median(ns)) - 0.5 * np.log(256 * 8192)) < 0.15
    assert {r.d for r in reqs} == set(range(2, 13))
    assert {r.p for r in reqs} == {1.5, 1.95, 2.0} and {r.delta for r in reqs} == {1e-8, 1e-6}
    fit_ids = set()
    for r in reqs:
        if r.kind == "fit":
            fit_ids.add(r.rid)
        else:
            assert r.target in fit_ids            # a predict names an earlier fit


def test_request_data_shapes():
    r = inputs.serving_stream(count=3)[0]
    x, y, th, xs = inputs.request_data(r, N=50)
    assert x.shape == (r.n, r.d) and y.shape == (r.n,) and th.shape == (32, r.d) and xs.shape == (50, r.d)
    x2, _, th2, _ = inputs.request_data(r, N=50)
    assert np.array_equal(x, x2) and np.array_equal(th, th2)
