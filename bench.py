"""Benchmark: profile -2logL evaluations per second at n = 4000.

Workload (one "step"): -2logL, mu_hat, sigma2_hat and log|R| at T = 256
theta candidates (a multi-start population, log10 theta ~ U[-2, 1]^6) on a
seeded random Latin hypercube of n = 4000 points in d = 6 with the smooth
synthetic response sum_k sin(2 pi x_k)/k + 0.1 sum_k x_k^2, p = 1.95,
delta = 1e-7 -- the shape of the paper's Example 2 (Hartman-6, n = 4064,
p = 1.95, Section 4), whose test function is not used.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
                  [--impl gp|reference]

--impl gp (default) times the CUDA library (inputs resident in HBM, CUDA
events on the library's stream, max over ranks; each rank evaluates its own
256 candidates: weak scaling, no collective on the data path).  The line
also carries the end-to-end number through the host-buffer C entry point,
the roofline of the dominant kernel, the SM clocks seen during the timed
region, and the CPU oracle timed on a bounded sample on the host cores.
--impl reference times the CPU oracle itself, on rank 0 only.
"""
import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1203_1269_gb300 import inputs  # noqa: E402

METRIC = "GP -2logL evals/s at n=4000 (d=6, T=256 theta batch)"
UNIT = "evals/s"
NB = 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def variance_flops(n, N, nb=NB):
    """The kriging variance's solve v = L^-1 r for N points: n^2 / 2
    multiply-adds per point (the method's work, 2 flops each), and the split
    GEMMs the tensor-core pass executes for it (per 128-point block and tile
    row J: the update, 15 slice products x 2 x 128^2 x 128 J, and the
    diagonal step, 28 products x 2 x 128^3)."""
    nt = -(-n // nb)
    blocks = -(-N // nb)
    executed = blocks * (15 * 2 * nb ** 3 * nt * (nt - 1) // 2 + 28 * 2 * nb ** 3 * nt)
    return float(n) * n * N, float(executed)


def update_flops(n, nb=NB):
    """Algorithmic flops of the trailing updates of one Cholesky (real rows
    only): sum over block steps of nb * m (m + 1), m = rows below the panel."""
    f = 0
    J = 0
    while (J + 1) * nb < n:
        m = n - (J + 1) * nb
        f += nb * m * (m + 1)
        J += 1
    return float(f)


def chol_flops(n):
    return n ** 3 / 3.0


def fp64_dgemm_tflops(dev, m=4096, reps=5):
    """The FP64 peak this GPU reaches in a dense library GEMM (cuBLAS DGEMM
    through torch.matmul, best of `reps`, CUDA events): the denominator of
    the FP64 path's roofline, measured in the same run."""
    import torch
    a = torch.randn(m, m, dtype=torch.float64, device=dev)
    b = torch.randn(m, m, dtype=torch.float64, device=dev)
    a @ b
    torch.cuda.synchronize(dev)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * m ** 3 / (best / 1e3) / 1e12


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# The workloads a step can run: the benchmark (the Hartman-shaped n = 4000
# batch) and, for measurement beside it, the batched n = 2048 case and the
# large n = 16384 instance of the other configurations.
WORKLOADS = ("hartman", "batched", "large")


def workload_for_rank(rank, n=4000, T=256, name="hartman"):
    if name == "batched":
        w = inputs.batched_split()
        seed = inputs.BASE_SEED + 2
    elif name == "large":
        w = inputs.large_instance()
        seed = inputs.BASE_SEED + 3
    else:
        w = inputs.hartman_shape(n=n, T=T)
        seed = inputs.BASE_SEED + 1
    if rank > 0:
        w.thetas = inputs.log_uniform_thetas(inputs.rng(seed + 1000 * rank), w.T, w.d)
    return w


def _code_only(text):
    """Source text without comments and with whitespace collapsed: what the
    compiler sees, so that editing a comment keeps a capture valid."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1203_1269_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def stored_traffic(kernel, src_files, units_per_launch=None):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on
    the current source of that kernel (else None).  A capture of a smaller
    case stores bytes per tile, scaled here by the tiles one launch updates."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except OSError:
        return None
    ent = table.get(kernel)
    if not ent or ent.get("source_hash") != kernel_source_hash(src_files):
        return None
    if "bytes_per_launch" in ent:
        return ent["bytes_per_launch"]
    if "bytes_per_tile" in ent and units_per_launch:
        return ent["bytes_per_tile"] * units_per_launch
    return None


def cpu_baseline_sample(w, max_theta=None, timeout_s=60.0):
    """The oracle, as it stands, on a bounded sample of the workload's
    candidates, spread over the host cores by its OpenMP loop."""
    import oracle
    cores = oracle.num_threads()
    k = min(w.T, max_theta or cores)
    t0 = time.perf_counter()
    out, st = oracle.nll_batch(w.x, w.y, w.thetas[:k], w.p, w.delta)
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} of the {w.T} candidates at n={w.n}, d={w.d} "
                      f"(one single-threaded evaluation per core, {dt:.1f} s)",
            "seconds": dt}, out, st


def oracle_errors(o_out, o_st, mixed, fp64):
    """Both GPU arms against the oracle on the oracle's own sample (the
    first candidates of the batch): relative error of -2logL per candidate."""
    k = len(o_st)
    mix = mixed["nll"][:k].cpu().numpy()
    f64 = fp64["nll"][:k].cpu().numpy()
    rows, wm, wf = [], 0.0, 0.0
    for t in range(k):
        if o_st[t] != 0:
            continue
        ref = o_out[t, 0]
        em = abs(mix[t] - ref) / abs(ref)
        ef = abs(f64[t] - ref) / abs(ref)
        wm, wf = max(wm, em), max(wf, ef)
        rows.append([t, float(f"{em:.3g}"), float(f"{ef:.3g}")])
    return {"candidates": k, "mixed_max_rel_err_nll": wm, "fp64_max_rel_err_nll": wf,
            "per_candidate_t_mixed_fp64": rows}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    w = workload_for_rank(0, args.n, args.T, args.workload)
    import oracle
    cores = oracle.num_threads()
    k = max(1, min(w.T, cores))
    for _ in range(args.warmup):
        oracle.nll_batch(w.x, w.y, w.thetas[:1], w.p, w.delta)
    times = []
    for s in range(args.steps):
        sel = w.thetas[(s * k) % w.T:(s * k) % w.T + k]
        t0 = time.perf_counter()
        oracle.nll_batch(w.x, w.y, sel, w.p, w.delta)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = k * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "d": w.d, "T": w.T, "p": w.p,
                       "delta": w.delta, "sample_per_step": k},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{k} candidates per step at n={w.n}, d={w.d}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gp(args):
    import torch
    import torch.distributed as dist
    from paper_1203_1269_gb300 import gp

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = workload_for_rank(rank, args.n, args.T, args.workload)
    prec = args.prec
    ctx = gp.Context(local)
    f64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x, y, th = f64(w.x), f64(w.y), f64(w.thetas)
    out = None

    def step():
        nonlocal out
        out = ctx.nll_batch(x, y, th, w.p, w.delta, prec, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    ok = int((st == 0).sum())

    # ---- timed region: device-resident inputs --------------------------------
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ctx.set_timing(True)
    ctx.phase_times()  # reset
    launches0 = ctx.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    phases = ctx.phase_times()
    ctx.set_timing(False)
    total_ms = t0.elapsed_time(t1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = world * w.T * args.steps / (total_ms / 1e3)

    # ---- roofline of the dominant kernel ------------------------------------
    pk, pk_src = peaks()
    dom = max(("assemble", "potrf", "trsm", "update", "solve", "split"), key=lambda k: phases[k][0])
    if prec == "fp64":
        upd_ms, upd_n = phases["update"]
        flops = update_flops(w.n) * w.T * args.steps
        achieved = flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None
        fp64_peak = fp64_dgemm_tflops(dev)
        roof = {"kernel": "k_update_f64", "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": (achieved / fp64_peak) if achieved else None,
                "traffic": stored_traffic("k_update_f64", ["k_chol_f64.cu"]),
                "peak_source": "FP64 dense, measured in this run: cuBLAS DGEMM (torch.matmul, "
                               "4096^3, best of 5, CUDA events)",
                "launches_timed": upd_n, "avg_launch_ms": upd_ms / max(upd_n, 1),
                "algorithmic_flops_per_launch": flops / max(upd_n, 1)}
    else:
        upd_ms, upd_n = phases["update"]
        opts = ctx.options()
        s = opts["slices"]
        prods = s * (s + 1) // 2
        nt = (w.n + NB - 1) // NB
        tiles = sum(m * (m + 1) // 2 for m in range(1, nt))          # trailing tiles per instance
        peak = pk["bf16_tflops_sustained"]
        # the method's own work: the trailing updates of one Cholesky of the n
        # real rows (update_flops), each executed as `prods` bf16 slice
        # products of the same shape
        alg_flops = update_flops(w.n) * prods * w.T * args.steps
        exec_flops = float(tiles) * prods * 2 * NB ** 3 * w.T * args.steps
        achieved = alg_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None
        executed = exec_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None
        # one unit = one 128 x 128 tile updated by one 128-wide panel; a launch
        # updates tiles * T * steps / launches of them on average (the fused
        # launches apply two panels per tile)
        units = tiles * w.T * args.steps / max(upd_n, 1)
        roof = {"kernel": "k_split_gemm<update>", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": stored_traffic("k_split_gemm<update>", ["k_gemm.cu", "mixed_common.cuh"], units),
                "units_per_launch": units,
                "algorithmic_bytes_per_launch": units * NB * NB * 8,
                "peak_source": ("bf16 dense sustained, measured (MEASURED_PEAKS.json)" if pk_src == "measured"
                                else "bf16 dense sustained, fallback (1.7 PFLOP/s; MEASURED_PEAKS.json absent)"),
                "flops_counted": f"algorithmic: the trailing updates of the {w.n} real rows "
                                 f"(sum over block steps of 128 m (m + 1)) x {prods} slice products",
                "frac_executed": (executed / peak) if executed else None,
                "executed_flops_note": f"executed: {tiles} whole 128x128 tiles per instance x {prods} "
                                       f"products x 2*128^3; the padded rows and the upper halves of the "
                                       f"diagonal tiles are {100.0 * (1.0 - alg_flops / exec_flops):.1f}% of it",
                "launches_timed": upd_n, "avg_launch_ms": upd_ms / max(upd_n, 1),
                "flops_per_launch": alg_flops / max(upd_n, 1),
                "fp64_equivalent_tflops": update_flops(w.n) * w.T * args.steps / (upd_ms / 1e3) / 1e12}

    # ---- end to end through the host-buffer entry point ---------------------
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    hx = torch.from_numpy(w.x.copy()).pin_memory()
    hy = torch.from_numpy(w.y.copy()).pin_memory()
    hth = torch.from_numpy(w.thetas.copy()).pin_memory()
    hout = dict(nll=torch.empty(w.T, dtype=torch.float64).pin_memory(),
                mu=torch.empty(w.T, dtype=torch.float64).pin_memory(),
                sigma2=torch.empty(w.T, dtype=torch.float64).pin_memory(),
                logdet=torch.empty(w.T, dtype=torch.float64).pin_memory(),
                status=torch.empty(w.T, dtype=torch.int32).pin_memory())
    ctx.nll_batch_host(hx, hy, hth, w.p, w.delta, prec, out=hout)
    if world > 1:
        dist.barrier()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.nll_batch_host(hx, hy, hth, w.p, w.delta, prec, out=hout)
    e2e_s = time.perf_counter() - te
    if world > 1:
        tt = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    h2d = (w.x.size + w.y.size + w.thetas.size) * 8
    d2h = w.T * (4 * 8 + 4)
    e2e = {"value": world * w.T * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    # ---- secondary precision (the other arm of the metric) -------------------
    other = None
    fp64_out = None
    if args.compare and prec == "mixed":
        o = ctx.nll_batch(x, y, th, w.p, w.delta, "fp64")
        torch.cuda.synchronize()
        ctx.set_timing(True)
        ctx.phase_times()
        a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.compare_steps):
            o = ctx.nll_batch(x, y, th, w.p, w.delta, "fp64", out=o)
        a1.record(stream)
        torch.cuda.synchronize()
        ph64 = ctx.phase_times()
        ctx.set_timing(False)
        ms = a0.elapsed_time(a1)
        fp64_out = o
        ref = o["nll"].cpu().numpy()
        got = out["nll"].cpu().numpy()
        # the tolerance applies where cond_1(R) <= 1e8: take the library's own
        # condition estimates (an untimed split-precision pass with them)
        cnd = ctx.nll_batch(x, y, th, w.p, w.delta, "mixed", cond=True)["cond"].cpu().numpy()
        fin = np.isfinite(ref) & np.isfinite(got)
        rel = np.abs(got[fin] - ref[fin]) / np.abs(ref[fin])
        wc = cnd[fin] <= 1e8
        # beyond cond_1 = 1e8 the error is reported against the rounding bound
        # n cond_1 u (u = 2^-53) of a factorisation in double, in absolute
        # terms: log|R| and n log Q carry absolute errors, and -2logL itself
        # may be close to zero
        absd = np.abs(got[fin] - ref[fin])
        ratio = absd / (w.n * cnd[fin] * 2.0 ** -53)
        upd64_ms = ph64["update"][0]
        upd64 = update_flops(w.n) * w.T * args.compare_steps / (upd64_ms / 1e3) / 1e12 if upd64_ms else None
        dg = fp64_dgemm_tflops(dev)
        other = {"prec": "fp64", "value": world * w.T * args.compare_steps / (ms / 1e3),
                 "steps": args.compare_steps,
                 "update_fp64_tflops": upd64, "fp64_dgemm_tflops_measured": dg,
                 "update_frac_of_dgemm": (upd64 / dg) if upd64 else None,
                 "mixed_vs_fp64_rel_err_nll": {
                     "max": float(rel.max()) if rel.size else None,
                     "median": float(np.median(rel)) if rel.size else None,
                     "max_where_cond1_le_1e8": float(rel[wc].max()) if wc.any() else None,
                     "candidates_cond1_le_1e8": int(wc.sum()),
                     "cond1_range": [float(np.nanmin(cnd)), float(np.nanmax(cnd))],
                     "max_abs": float(absd.max()) if absd.size else None,
                     "max_abs_err_over_n_cond1_u": float(ratio.max()) if ratio.size else None,
                     "per_candidate_cond1_rel_abs": [[float(f"{c:.3g}"), float(f"{e:.3g}"), float(f"{a:.3g}")]
                                                     for c, e, a in zip(cnd[fin], rel, absd)]}}

    # ---- kriging at the best candidate (the large instance's N = 1e5 points) --
    kriging = None
    if args.workload == "large" and w.xs is not None:
        st_h = out["status"].cpu().numpy()
        nll_h = out["nll"].cpu().numpy()
        okc = np.where(st_h == 0)[0]
        best = int(okc[np.argmin(nll_h[okc])])
        torch.cuda.synchronize()
        k0 = time.perf_counter()
        model = ctx.fit(x, y, th[best].contiguous(), w.p, w.delta, "fp64")
        torch.cuda.synchronize()
        t_fit = time.perf_counter() - k0
        xs = f64(w.xs)
        ctx.predict(model, xs[:1000])
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True); p1 = torch.cuda.Event(enable_timing=True)
        p2 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        ctx.predict(model, xs, want_var=False)
        p1.record(stream)
        ctx.predict(model, xs)
        p2.record(stream)
        torch.cuda.synchronize()
        t_mean, t_var = p0.elapsed_time(p1) / 1e3, p1.elapsed_time(p2) / 1e3
        method, executed = variance_flops(w.n, int(xs.shape[0]))
        pk, _ = peaks()
        t_tc = t_var - t_mean   # the tables and the tensor-core pass (r is formed by both calls)
        # the double-float substitution on the FP32 pipes, on the first 1e4 points
        ctx.set_options(predict_tc=0)
        q0 = torch.cuda.Event(enable_timing=True); q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        ctx.predict(model, xs[:10000])
        q1.record(stream)
        torch.cuda.synchronize()
        ctx.set_options(predict_tc=1)
        kriging = {"N": int(xs.shape[0]), "candidate": best, "fit_s": t_fit,
                   "mean_only_s": t_mean, "mean_and_variance_s": t_var,
                   "variance_solve": {"tensor_core_pass_s": t_tc,
                                      "method_tflops": method / t_tc / 1e12,
                                      "executed_split_tflops": executed / t_tc / 1e12,
                                      "executed_frac_of_sustained_bf16": executed / t_tc / 1e12 / pk["bf16_tflops_sustained"],
                                      "flops_counted": "method: n^2 N (v = L^-1 r); executed: the split GEMMs "
                                                       "(15 products in the updates, 28 in the diagonal steps)"},
                   "fp32_pipes_mean_and_variance_1e4_points_s": q0.elapsed_time(q1) / 1e3}
        model.free()

    cpu = None
    if args.workload == "large":
        pass   # one oracle evaluation at n = 16384 takes minutes: no bounded sample
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, o_out, o_st = cpu_baseline_sample(w)
        if other is not None:
            other["vs_oracle"] = oracle_errors(o_out, o_st, out, fp64_out)

    if rank == 0:
        pct = lambda q: float(np.percentile(step_ms, q))
        metric = METRIC if args.workload == "hartman" else \
            f"GP -2logL evals/s at n={w.n} (d={w.d}, T={w.T} theta batch)"
        line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == "fp64" else "bf16-split/f64",
                "data": "synthetic",
                "config": {"workload": w.name, "n": w.n, "d": w.d, "T": w.T, "p": w.p,
                           "delta": w.delta, "prec": prec, "parallelism": f"replicas{world}",
                           "l2": "no flush: the batch's factor storage "
                                 f"({w.T * ((w.n + NB - 1) // NB) * ((w.n + NB - 1) // NB + 1) // 2 * NB * NB * 8 / 1e9:.1f} GB) "
                                 "exceeds L2 (129 MB)"},
                "latency_ms": {"p50": pct(50), "p99": pct(99), "unit": f"ms per {w.T}-candidate batch"},
                "statuses_ok": ok,
                "roofline": roof, "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()
                                                         if v[1]},
                "gpu_launches": launches, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
        if other:
            line["compare"] = other
        if kriging:
            line["kriging"] = kriging
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    ctx.close()
    return 0


def run_kriging(args):
    """Kriging alone: the large instance's design (random Latin hypercube,
    d = 10, p = 1.9, delta = 1e-6) at n = --n (16384 unless given), its first
    candidate fitted in FP64, then gp_predict at --points uniform test points:
    means only, means and variances (the variance's solve on the tensor
    cores), each timed with CUDA events after --warmup calls."""
    import torch
    from paper_1203_1269_gb300 import gp
    n = args.n if args.n != 4000 else 16384
    w = inputs.large_instance(n=n, T=1, N=args.points)
    ctx = gp.Context(0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    model = ctx.fit(dev(w.x), dev(w.y), dev(w.thetas[0]), w.p, w.delta, "fp64")
    xs = dev(w.xs)
    stream = torch.cuda.current_stream()

    def timed(want_var):
        for _ in range(args.warmup):
            ctx.predict(model, xs, want_var=want_var)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            out = ctx.predict(model, xs, want_var=want_var)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / args.steps, out

    t_mean, _ = timed(False)
    t_var, (_, s2) = timed(True)
    method, executed = variance_flops(n, args.points)
    pk, _ = peaks()
    t_tc = t_var - t_mean
    print(json.dumps({"metric": f"kriging points/s (mean and variance) at n={n}, d={w.d}",
                      "value": args.points / t_var, "unit": "points/s", "higher_is_better": True,
                      "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                      "config": {"workload": f"kriging n={n} d={w.d} N={args.points}", "p": w.p, "delta": w.delta},
                      "mean_only_s": t_mean, "mean_and_variance_s": t_var,
                      "variance_nan": int(torch.isnan(s2).sum()),
                      # the pass is the difference of two timings: too short a pass to
                      # resolve (tiny n or N) reports no rate
                      "variance_solve": {"tensor_core_pass_s": t_tc,
                                         "method_tflops": method / t_tc / 1e12 if t_tc > 0 else None,
                                         "executed_split_tflops": executed / t_tc / 1e12 if t_tc > 0 else None,
                                         "executed_frac_of_sustained_bf16":
                                             executed / t_tc / 1e12 / pk["bf16_tflops_sustained"] if t_tc > 0 else None}}))
    model.free()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gp", choices=["gp", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip timing the FP64 arm beside the mixed one")
    ap.add_argument("--compare-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=4000, help="design size (profiling cases only)")
    ap.add_argument("--T", type=int, default=256, help="candidates per step (profiling cases only)")
    ap.add_argument("--workload", default="hartman", choices=WORKLOADS,
                    help="hartman: the benchmark (n = 4000, d = 6, T = 256); batched: n = 2048, "
                         "d = 8, T = 1024; large: n = 16384, d = 10, T = 32 with kriging at 1e5 points")
    ap.add_argument("--kriging-only", action="store_true",
                    help="fit one candidate of the large instance at --n (default 16384) design points "
                         "and time gp_predict at --points test points; one JSON line")
    ap.add_argument("--points", type=int, default=100000, help="test points of --kriging-only")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.kriging_only:
        return run_kriging(args)
    return run_gp(args)


if __name__ == "__main__":
    sys.exit(main())
