"""GPU test of gp_nll_batch_noalloc, the entry point for callers that cannot
let the library allocate device memory (its scratch is a fixed array inside
the library).  Named to run last, so that a run stopping at the first failure
has run every other test first.

Checks, through the C ABI: two calls in a row give gp_nll_batch's double
precision results bit for bit (both run the same per-candidate kernels, so
any difference, even in the last bits, would mean a layout or offset error),
a batch larger than one round of the scratch array is handled, a small n
after the largest one reads nothing the larger call left behind, and an n
that does not fit is rejected with GP_ENOMEM.
"""
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


def same_bits(got, ref):
    assert torch.equal(got["status"], ref["status"])
    for k in ("nll", "mu", "sigma2", "logdet"):
        a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), k


@pytest.mark.parametrize("n,T", [(200, 64), (1000, 40)])
def test_noalloc_matches_nll_batch_twice(ctx, n, T):
    # (1000, 40): 7 candidates fit the array at n = 1000, so the batch takes six rounds
    w = inputs.hartman_shape(n=n, d=6, T=T)
    x, y, th = dev(w.x), dev(w.y), dev(w.thetas)
    ref = ctx.nll_batch(x, y, th, w.p, w.delta, "fp64")
    for _ in range(2):
        got = ctx.nll_batch_noalloc(x, y, th, w.p, w.delta)
        torch.cuda.synchronize()
        same_bits(got, ref)


def test_noalloc_small_after_largest(ctx):
    """n = 2816 fills the array with one candidate; an n = 200 call after it on
    the same stream must give the same bits as before it (every buffer a call
    reads, it writes first)."""
    small = inputs.hartman_shape(n=200, d=6, T=8)
    big = inputs.hartman_shape(n=2816, d=6, T=2)
    xs, ys, ts = dev(small.x), dev(small.y), dev(small.thetas)
    ref = ctx.nll_batch(xs, ys, ts, small.p, small.delta, "fp64")
    before = ctx.nll_batch_noalloc(xs, ys, ts, small.p, small.delta)
    big_ref = ctx.nll_batch(dev(big.x), dev(big.y), dev(big.thetas), big.p, big.delta, "fp64")
    big_got = ctx.nll_batch_noalloc(dev(big.x), dev(big.y), dev(big.thetas), big.p, big.delta)
    after = ctx.nll_batch_noalloc(xs, ys, ts, small.p, small.delta)
    torch.cuda.synchronize()
    same_bits(before, ref)
    same_bits(big_got, big_ref)
    same_bits(after, ref)


def test_noalloc_rejects_n_beyond_the_array(ctx):
    from paper_1203_1269_gb300 import gp
    n = 2817
    x = dev(np.random.default_rng(1).random((n, 2)))
    y = dev(np.zeros(n))
    with pytest.raises(gp.GPError) as err:
        ctx.nll_batch_noalloc(x, y, dev([[1.0, 1.0]]), 2.0, 1e-6)
    assert err.value.code == gp.GP_ENOMEM
    assert "2816" in str(err.value)
