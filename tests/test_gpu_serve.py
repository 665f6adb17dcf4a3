"""GPU test of the continuous-batching server: a stream of fit and predict
requests of different n, d, p and delta runs on four concurrent CUDA streams
under an HBM budget; every result equals the result of the same request run
alone, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _stream():
    from paper_1203_1269_gb300 import inputs
    return inputs.serving_stream(count=14, rate=1e6, n_lo=200, n_hi=700, seed=4242)


def test_results_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import serve
    reqs = _stream()
    assert {r.kind for r in reqs} == {"fit", "predict"}
    mix = serve.Server(workers=4, budget_bytes=8 << 30, N_pred=200)
    res_mix = mix.run(reqs, realtime=False)
    mix.close()
    alone = {}
    for r in reqs:
        srv = serve.Server(workers=1, budget_bytes=8 << 30, N_pred=200)
        needed = [q for q in reqs if q.rid == r.target] + [r] if r.kind == "predict" else [r]
        alone[r.rid] = srv.run(needed, realtime=False)[r.rid]
        srv.close()
    for r in reqs:
        a, b = res_mix[r.rid], alone[r.rid]
        assert a.status == b.status == 0, (r.rid, a.status, b.status)
        if r.kind == "fit":
            assert a.best == b.best
            assert np.array_equal(a.nll, b.nll)
            assert a.mu == b.mu and a.sigma2 == b.sigma2
        else:
            assert np.array_equal(a.yhat, b.yhat)
            assert np.array_equal(a.s2, b.s2)
    lat = [x.done - x.arrival for x in res_mix.values()]
    assert all(t > 0 for t in lat)


def test_budget_forces_release_and_refit():
    """A budget that holds about one factor: earlier fits are released and
    the predictions against them refit first, with unchanged results."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_1269_gb300 import serve
    reqs = _stream()
    big = serve.Server(workers=2, budget_bytes=8 << 30, N_pred=200)
    ref = big.run(reqs, realtime=False)
    big.close()
    small = serve.Server(workers=1, budget_bytes=96 << 20, N_pred=200)
    got = small.run(reqs, realtime=False)
    small.close()
    for r in reqs:
        if r.kind == "predict":
            assert np.array_equal(got[r.rid].yhat, ref[r.rid].yhat)
    assert sum(x.refit for x in got.values()) >= 1
