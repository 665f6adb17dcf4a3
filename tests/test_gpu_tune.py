"""Launch-shape options of the split path and the autotuner (gp_autotune)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1203_1269_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("nll", "mu", "sigma2", "logdet", "status")


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


def case(seed=601, n=700, d=3, T=12):
    g = np.random.default_rng(seed)
    x = inputs.random_lhd(g, n, d)
    y = inputs.y_sinsum(x)
    th = inputs.log_uniform_thetas(g, T, d, lo=-0.5, hi=1.0)
    return x, y, th, 1.95, 1e-6


@pytest.mark.parametrize("fuse", [1, 0])
def test_shape_options_leave_results_unchanged(ctx, fuse):
    """64-column update tiles and 32-column assembly parts run the same
    arithmetic in the same order as the defaults: identical results."""
    x, y, th, p, delta = case()
    X, Y, TH = dev(x), dev(y), dev(th)
    base_opts = ctx.options()
    try:
        ctx.set_options(fuse_panels=fuse, update_tile=128, assemble_cols=16)
        ref = ctx.nll_batch(X, Y, TH, p, delta, "mixed")
        variants = [dict(update_tile=64), dict(assemble_cols=32), dict(update_tile=64, assemble_cols=32)]
        for kw in variants:
            ctx.set_options(fuse_panels=fuse, update_tile=kw.get("update_tile", 128),
                            assemble_cols=kw.get("assemble_cols", 16))
            got = ctx.nll_batch(X, Y, TH, p, delta, "mixed")
            for k in KEYS:
                assert np.array_equal(host(got[k]), host(ref[k]), equal_nan=True), (kw, k)
    finally:
        ctx.set_options(**base_opts)


def test_autotune_keeps_fastest(ctx):
    x, y, th, p, delta = case(seed=602, n=900, T=16)
    X, Y, TH = dev(x), dev(y), dev(th)
    base_opts = ctx.options()
    try:
        trials, chosen = ctx.autotune(X, Y, TH, p, delta, "mixed", reps=2)
        assert len(trials) == 8
        best = min(trials, key=lambda t: t["ms"])
        for k in ("update_tile", "fuse_panels", "assemble_cols"):
            assert chosen[k] == best[k]
        print("\nautotune n=900 T=16:", [(t["update_tile"], t["fuse_panels"], t["assemble_cols"],
                                          round(t["ms"], 3)) for t in trials])
        # the tuned context still meets the split path's tolerance
        ref, st = oracle.nll_batch(x, y, th, p, delta, want_cond=True)
        res = ctx.nll_batch(X, Y, TH, p, delta, "mixed")
        ok = (st == 0) & (ref[:, 6] <= 1e8)
        rel = np.abs(host(res["nll"])[ok] - ref[ok, 0]) / np.abs(ref[ok, 0])
        assert ok.any() and rel.max() <= 1e-6
    finally:
        ctx.set_options(**base_opts)


def test_autotune_rejects_fp64(ctx):
    from paper_1203_1269_gb300 import gp
    x, y, th, p, delta = case(T=2)
    with pytest.raises(gp.GPError) as e:
        ctx.autotune(dev(x), dev(y), dev(th), p, delta, "fp64")
    assert e.value.code == gp.GP_ENOTSUP


def test_shape_option_validation(ctx):
    from paper_1203_1269_gb300 import gp
    base_opts = ctx.options()
    try:
        for kw in (dict(update_tile=96), dict(assemble_cols=8), dict(update_tile=64, update_groups=3, fuse_panels=0)):
            with pytest.raises(gp.GPError):
                ctx.set_options(**kw)
    finally:
        ctx.set_options(**base_opts)
