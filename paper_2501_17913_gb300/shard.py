"""Trajectory sharding across ranks (one process per GPU).

Trajectories are independent (TJM Sec. "Tensor jump method": the process is
embarrassingly parallel), and each draws its random numbers from a Philox
counter keyed by its GLOBAL id, so splitting the ids over ranks changes no
result.  The only exchange is the final merge of per-(time, observable)
moments, one all-reduce of three small arrays.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_total: int, rank: int, world: int):
    """Contiguous global trajectory ids [first, first + count) of this rank."""
    base, extra = divmod(n_total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def _allreduce_sum(arr, group=None):
    import torch
    import torch.distributed as dist
    buf = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64).ravel().copy())
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            buf = buf.cuda()
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
        buf = buf.cpu()
    return buf.numpy().reshape(np.shape(arr))


def merge_ensemble(per_traj_local, group=None):
    """Mean and standard error over the trajectories of all ranks, two-pass.

    First all-reduce (sum x, count) for the global mean, then the sum of squared
    deviations from it, so the variance does not suffer the cancellation of
    sum x^2 - N mean^2.  per_traj_local: [n_local][times][obs].
    """
    x = np.asarray(per_traj_local, dtype=np.float64)
    shp = x.shape[1:]
    first = _allreduce_sum(np.concatenate([x.sum(axis=0).ravel(), [float(x.shape[0])]]), group)
    n = first[-1]
    mean = first[:-1].reshape(shp) / n
    m2 = _allreduce_sum(((x - mean) ** 2).sum(axis=0), group)
    return mean, np.sqrt(m2 / max(n - 1.0, 1.0) / n)


def job_rate(units, ms):
    """Whole-job throughput across ranks: the units all ranks processed over the slowest rank's time
    (the job ends when its last rank does).  Returns (units per second, slowest time in ms).
    Without an initialised process group this is the local rate."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units / (ms / 1000.0), ms
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return float(u.item()) / (t_max / 1000.0), t_max


class PeerFailure(RuntimeError):
    """A rank did not report in time: it failed, left or never joined."""


def report_alive(store, rank: int, tag: str):
    """Record in the shared key-value store that this rank reached `tag` (e.g. the end of a step)."""
    store.set("%s/%d" % (tag, rank), "1")


def wait_peers(store, world: int, tag: str, timeout_s: float):
    """Block until every rank has reported `tag`; raise PeerFailure naming the missing ranks after
    timeout_s.  Ranks call this between steps, before their next launch, so a rank that died is
    noticed on the host and no kernel or collective is left waiting on it."""
    import time
    deadline = time.monotonic() + timeout_s
    missing = list(range(world))
    while True:
        missing = [r for r in missing if not store.check(["%s/%d" % (tag, r)])]
        if not missing:
            return
        if time.monotonic() >= deadline:
            raise PeerFailure("ranks %s did not reach %r within %.1f s" % (missing, tag, timeout_s))
        time.sleep(0.05)
