"""GPU test of gp_nll_batch_noalloc, the entry point for callers that cannot
let the library allocate device memory (its scratch is a fixed array inside
the library).  Named to run last, so that a run stopping at the first failure
has run every other test first.

Checks, through the C ABI: two calls in a row agree with gp_nll_batch in
double precision within the tolerance of the other FP64 tests (1e-9 relative
on -2logL, mu_hat, sigma2_hat), a batch larger than one round of the scratch
array is handled, and an n that does not fit is rejected with GP_ENOMEM.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1203_1269_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import gp
    return gp.Context(0)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def close(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return np.all(np.abs(a[fin] - b[fin]) <= TOL * np.maximum(1.0, np.abs(b[fin])))


@pytest.mark.parametrize("n,T", [(200, 64), (1000, 40)])
def test_noalloc_matches_nll_batch_twice(ctx, n, T):
    # (1000, 40): 7 candidates fit the array at n = 1000, so the batch takes six rounds
    w = inputs.hartman_shape(n=n, d=6, T=T)
    x, y, th = dev(w.x), dev(w.y), dev(w.thetas)
    ref = ctx.nll_batch(x, y, th, w.p, w.delta, "fp64")
    for _ in range(2):
        got = ctx.nll_batch_noalloc(x, y, th, w.p, w.delta)
        torch.cuda.synchronize()
        assert torch.equal(got["status"], ref["status"])
        for k in ("nll", "mu", "sigma2", "logdet"):
            assert close(got[k], ref[k]), k


def test_noalloc_rejects_n_beyond_the_array(ctx):
    from paper_1203_1269_gb300 import gp
    n = 2817
    x = dev(np.random.default_rng(1).random((n, 2)))
    y = dev(np.zeros(n))
    with pytest.raises(gp.GPError) as err:
        ctx.nll_batch_noalloc(x, y, dev([[1.0, 1.0]]), 2.0, 1e-6)
    assert err.value.code == gp.GP_ENOMEM
    assert "2816" in str(err.value)
