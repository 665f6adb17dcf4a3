"""Continuous-batching request server over libgp.

Requests are fits (the -2logL of a request's 32 theta candidates and the fit
of the best one from its own factor, gp_fit_batch, whose factor then stays
resident on the device) and predictions (gp_predict against a resident fit).
Everything runs at the server's precision: with "mixed" the resident factors
are the split-precision ones (kriging variances to about cond(R) 2^-40), with
"fp64" double ones.  Work runs on
`workers` CUDA streams at once, one libgp context per stream, so requests of
different n and d overlap on the GPU.  A request is admitted as soon as a
stream is free and its device memory fits the HBM budget next to what is
already held (workspaces of the contexts plus resident factors); otherwise it
waits, and later requests that fit go ahead of it.  A prediction waits for
its fit.  When resident factors would exceed the budget, the least recently
used ones are released; a prediction against a released fit refits it at its
chosen theta first.

Every result depends only on its own request: each candidate's factorisation
and reductions run in a fixed order whatever else shares the GPU, so results
are identical alone and in the mix (tests/test_gpu_serve.py checks this).

    python -m paper_1203_1269_gb300.serve [--requests 2000] [--rate 200]
           [--workers 4] [--budget-gb 120] [--prec mixed]
"""
import argparse
import collections
import functools
import json
import threading
import time

import numpy as np
import torch

from . import gp, inputs

_MB = 1 << 20


FIT_CANDIDATES = 32   # theta candidates evaluated per fit request (inputs.request_data)


# The scheduler sizes every queued request at each pick: the library's figures
# depend only on these arguments (default options, no budget), so keep them.
@functools.lru_cache(maxsize=4096)
def eval_bytes(n, d, prec, T=FIT_CANDIDATES):
    """Workspace of gp_nll_batch for T candidates, as the library sizes it."""
    return gp.call_bytes("nll_batch", n, d, T, prec)


@functools.lru_cache(maxsize=4096)
def model_bytes(n, d):
    return gp.call_bytes("fit", n, d)


@functools.lru_cache(maxsize=4096)
def predict_bytes(n, d, N):
    return gp.call_bytes("predict", n, d, N)


class Result:
    __slots__ = ("rid", "kind", "arrival", "start", "done", "theta", "nll", "mu", "sigma2",
                 "best", "yhat", "s2", "status", "error", "refit", "t_eval", "t_fit", "t_pred")

    def __init__(self, rid, kind):
        self.rid, self.kind = rid, kind
        self.arrival = self.start = self.done = None
        self.theta = self.nll = self.mu = self.sigma2 = self.best = None
        self.yhat = self.s2 = None
        self.status = None
        self.error = None
        self.refit = False
        self.t_eval = self.t_fit = self.t_pred = 0.0


class Server:
    def __init__(self, workers=4, budget_bytes=120 * 1024 * _MB, prec="mixed", device=0, N_pred=1000):
        self.device = device
        self.prec = prec
        self.budget = budget_bytes
        self.N_pred = N_pred
        self.lock = threading.Condition()
        self.queue = collections.deque()
        self.results = {}
        self.models = collections.OrderedDict()   # rid -> (Model, theta, p, delta) in LRU order
        self.fit_done = {}                        # rid -> threading.Event
        self.worker_ws = [0] * workers
        self.in_flight = [0] * workers
        self.model_held = 0
        self.closed = False
        self.requests = {}                        # rid -> Request
        self.busy = [False] * workers
        self.ctxs = []
        self.streams = []
        for _ in range(workers):
            s = torch.cuda.Stream(device=device)
            self.streams.append(s)
            # the server admits by its own budget; each context may size its workspace freely
            self.ctxs.append(gp.Context(device, hbm_budget_bytes=0, stream=s))
        self.threads = [threading.Thread(target=self._work, args=(i,), daemon=True) for i in range(workers)]
        for t in self.threads:
            t.start()

    # -- accounting ----------------------------------------------------------
    def _held(self):
        return sum(self.worker_ws) + sum(self.in_flight) + self.model_held

    def _need(self, req):
        if req.kind == "fit":
            return eval_bytes(req.n, req.d, self.prec) + model_bytes(req.n, req.d)
        tgt = self.requests[req.target]
        return predict_bytes(tgt.n, tgt.d, self.N_pred) + model_bytes(tgt.n, tgt.d)

    # -- submission ----------------------------------------------------------
    def submit(self, req):
        with self.lock:
            self.requests[req.rid] = req
            r = Result(req.rid, req.kind)
            r.arrival = time.perf_counter()
            self.results[req.rid] = r
            if req.kind == "fit":
                self.fit_done[req.rid] = threading.Event()
            self.queue.append(req)
            self.lock.notify_all()

    def _pick(self, i):
        """Next admissible request for worker i (caller holds the lock)."""
        for k, req in enumerate(self.queue):
            if req.kind == "predict":
                ev = self.fit_done.get(req.target)
                if ev is None or not ev.is_set():
                    continue
            need = self._need(req)
            held_other = self._held() - self.worker_ws[i]
            if held_other + max(need, self.worker_ws[i]) <= self.budget or not any(self.busy):
                del self.queue[k]
                return req, need
        return None, 0

    def _evict_for(self, need, keep):
        """Release least recently used factors until `need` more bytes fit."""
        while self.models and self._held() + need > self.budget:
            rid, entry = next(iter(self.models.items()))
            if rid == keep:
                break
            self.models.pop(rid)
            self.model_held -= entry[0].bytes
            entry[0].free()

    # -- execution -----------------------------------------------------------
    def _work(self, i):
        ctx, stream = self.ctxs[i], self.streams[i]
        while True:
            with self.lock:
                while True:
                    if self.closed and not self.queue:
                        return
                    req, need = self._pick(i)
                    if req is not None:
                        break
                    self.lock.wait(timeout=0.05)
                self.busy[i] = True
                self.in_flight[i] = need
                self._evict_for(0, keep=req.target if req.kind == "predict" else -1)
            res = self.results[req.rid]
            res.start = time.perf_counter()
            try:
                with torch.cuda.stream(stream):
                    if req.kind == "fit":
                        self._fit(ctx, req, res)
                    else:
                        self._predict(ctx, req, res)
            except gp.GPError as e:
                res.status = e.code
                res.error = str(e)
            res.done = time.perf_counter()
            with self.lock:
                self.busy[i] = False
                self.in_flight[i] = 0
                self.worker_ws[i] = ctx.workspace_bytes()
                if req.kind == "fit":
                    self.fit_done[req.rid].set()
                self.lock.notify_all()

    def _device(self, a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).to(
            torch.device("cuda", self.device), non_blocking=False)

    def _fit(self, ctx, req, res):
        x, y, th, _ = inputs.request_data(req, self.N_pred)
        xd, yd, thd = self._device(x), self._device(y), self._device(th)
        # the candidates' -2logL and the fit of the best one, from its own
        # factor (gp_fit_batch: no second factorisation)
        t0 = time.perf_counter()
        out, best, model = ctx.fit_batch(xd, yd, thd, req.p, req.delta, self.prec)
        res.t_eval = time.perf_counter() - t0
        res.nll = out["nll"].cpu().numpy()
        st = out["status"].cpu().numpy()
        if model is None:
            res.status = int(st[0])
            return
        res.status = 0
        res.best, res.theta = best, th[best]
        res.mu, res.sigma2 = model.mu, model.sigma2
        with self.lock:
            self._evict_for(model.bytes, keep=req.rid)
            self.models[req.rid] = (model, th[best], req.p, req.delta)
            self.model_held += model.bytes

    def _predict(self, ctx, req, res):
        fit = self.results[req.target]
        src = self.requests[req.target]
        with self.lock:
            entry = self.models.get(req.target)
            if entry is not None:
                self.models.move_to_end(req.target)
        if fit.theta is None:
            res.status = fit.status if fit.status is not None else gp.GP_EINVAL
            return
        if entry is None:
            # released: refit at the chosen theta (same factor, same result)
            x, y, _, _ = inputs.request_data(src, self.N_pred)
            t0 = time.perf_counter()
            model = ctx.fit(self._device(x), self._device(y), self._device(fit.theta), src.p, src.delta, self.prec)
            res.t_fit = time.perf_counter() - t0
            res.refit = True
            with self.lock:
                self._evict_for(model.bytes, keep=req.target)
                entry = (model, fit.theta, src.p, src.delta)
                self.models[req.target] = entry
                self.model_held += model.bytes
        model = entry[0]
        xs = inputs.uniform_design(inputs.rng(req.seed), self.N_pred, src.d)
        t0 = time.perf_counter()
        yhat, s2 = ctx.predict(model, self._device(xs))
        res.yhat = yhat.cpu().numpy()
        res.t_pred = time.perf_counter() - t0
        res.s2 = s2.cpu().numpy()
        res.status = 0

    # -- driving a trace -----------------------------------------------------
    def run(self, requests, realtime=True):
        """Replay `requests` (arrival times in seconds) and wait for all of them."""
        t0 = time.perf_counter()
        for req in requests:
            if realtime:
                delay = t0 + req.arrival_s - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            self.submit(req)
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        for t in self.threads:
            t.join()
        torch.cuda.synchronize(self.device)
        return self.results

    def close(self):
        for m in list(self.models.values()):
            m[0].free()
        self.models.clear()
        for c in self.ctxs:
            c.close()


def summarize(results, requests):
    lat = np.array([r.done - r.arrival for r in results.values() if r.done is not None])
    span = max(r.done for r in results.values()) - min(r.arrival for r in results.values())
    fits = [r for r in results.values() if r.kind == "fit"]
    evals = sum(len(r.nll) for r in fits if r.nll is not None)
    return {"requests": len(results), "seconds": span, "req_per_s": len(results) / span,
            "evals_per_s": evals / span,
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "mean": float(lat.mean() * 1e3)},
            "refits": sum(r.refit for r in results.values()),
            "busy_s": {"evals_and_fits": sum(r.t_eval for r in results.values()),
                       "refits": sum(r.t_fit for r in results.values()),
                       "predicts": sum(r.t_pred for r in results.values())},
            "failed": sum(1 for r in results.values() if r.status not in (0, None)),
            "errors": dict(collections.Counter(f"{r.kind}: {r.error or r.status}" for r in results.values()
                                               if r.status not in (0, None)).most_common(5))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    reqs = inputs.serving_stream(count=args.requests, rate=args.rate)
    srv = Server(workers=args.workers, budget_bytes=int(args.budget_gb * (1 << 30)), prec=args.prec)
    res = srv.run(reqs)
    out = summarize(res, reqs)
    out.update({"workload": f"serving stream, {args.requests} requests, Poisson {args.rate}/s, "
                            "n log-uniform [256, 8192], d 2..12",
                "workers": args.workers, "prec": args.prec, "budget_gb": args.budget_gb})
    srv.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
