"""CPU test of the multi-rank path: candidates sharded over two gloo ranks,
each evaluated by the oracle, gathered, and compared with one process doing
the whole batch."""
import os
import socket

import numpy as np
import pytest

from paper_1203_1269_gb300 import shard


def test_shard_ranges_cover_exactly():
    for T in (1, 5, 256, 1023):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                a, b = shard.shard_range(T, world, r)
                got.extend(range(a, b))
                assert (b - a) in (T // world, T // world + 1)
            assert got == list(range(T))


def _evaluate(x, y, thetas, p, delta):
    import oracle
    out, st = oracle.nll_batch(x, y, thetas, p, delta)
    return {"nll": out[:, 0], "mu": out[:, 1], "sigma2": out[:, 2], "logdet": out[:, 3], "status": st}


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1203_1269_gb300 import inputs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = inputs.small_grid_fit(n=60, N=0)
    res = shard.nll_batch_sharded(_evaluate, w.x, w.y, w.thetas[:13], w.p, w.delta, world, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, {k: v.tolist() for k, v in res.items()}))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_match_single_process():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_1203_1269_gb300 import inputs
    w = inputs.small_grid_fit(n=60, N=0)
    ref = _evaluate(w.x, w.y, w.thetas[:13], w.p, w.delta)
    for r in (0, 1):
        for k in shard.FIELDS:
            assert np.array_equal(np.asarray(results[r][k]), np.asarray(ref[k])), (r, k)
