"""Candidates of a -2logL batch spread over ranks (one GPU per rank).

The candidates are independent (each is its own R(theta), factorisation and
solves), so the batch shards into contiguous blocks of theta rows with no
exchange on the data path.  When a caller wants every result on every rank
(an optimiser choosing the next population, say), `gather_results` moves the
T x 5 scalars -- the only exchange there is -- through torch.distributed on
the host side.
"""
import numpy as np


def shard_range(T: int, world: int, rank: int):
    """[start, stop) of rank's block; sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(T, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


FIELDS = ("nll", "mu", "sigma2", "logdet", "status")


def gather_results(local: dict, T: int, world: int, rank: int, dist=None):
    """All-gather each rank's block of results (numpy arrays keyed by FIELDS)
    into full length-T arrays on every rank."""
    if world == 1:
        return {k: np.asarray(local[k]) for k in FIELDS}
    import torch
    if dist is None:
        import torch.distributed as dist
    blocks = [shard_range(T, world, r) for r in range(world)]
    width = max(b1 - b0 for b0, b1 in blocks)
    a, b = blocks[rank]
    buf = torch.full((5, width), float("nan"), dtype=torch.float64)
    for i, k in enumerate(FIELDS):
        buf[i, : b - a] = torch.as_tensor(np.asarray(local[k], dtype=np.float64))
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = {k: np.empty(T, dtype=np.float64) for k in FIELDS}
    for r, (b0, b1) in enumerate(blocks):
        for i, k in enumerate(FIELDS):
            out[k][b0:b1] = parts[r][i, : b1 - b0].numpy()
    out["status"] = out["status"].astype(np.int32)
    return out


def nll_batch_sharded(evaluate, x, y, thetas, p, delta, world=1, rank=0, dist=None):
    """Evaluate this rank's block with `evaluate(x, y, thetas_block, p, delta)`
    (returning numpy arrays keyed by FIELDS) and gather the full batch."""
    T = len(thetas)
    a, b = shard_range(T, world, rank)
    local = evaluate(x, y, thetas[a:b], p, delta)
    return gather_results(local, T, world, rank, dist)
