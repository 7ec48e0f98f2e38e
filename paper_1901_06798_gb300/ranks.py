"""Several GPUs, one process each: sharding of independent scenarios and the
whole-job throughput rule.

An ensemble's scenarios share nothing but the bathymetry: each advances with
its own time step, patches and gauges.  So they partition across ranks with no
collective on the data path.  Rank r builds its own context holding scenarios
[lo, hi), steps it, and only the finished gauge records are gathered at the
end.  A uniform single-scenario grid does not partition this way (that would
need halo exchange every level step); there every rank runs a replica.

Everything here is host logic over ``torch.distributed`` (any backend); the
solver is whatever object the caller passes (the CUDA binding on a GPU machine).
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous balanced block [lo, hi) of n units for this rank; the first
    n % world ranks take one unit more."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_workload(w: dict, rank: int, world: int) -> tuple[dict, int, int]:
    """The part of workload ``w`` (the dict the workload generators return)
    that this rank advances: its scenarios, renumbered from 0."""
    n = w["cfg"].get("n_scenarios", 1)
    lo, hi = shard(n, rank, world)
    cfg = dict(w["cfg"], n_scenarios=max(hi - lo, 0))
    pick = lambda items: [(s - lo, *rest) for (s, *rest) in items if lo <= s < hi]
    return dict(w, cfg=cfg, eta=pick(w.get("eta", [])), uplift=pick(w.get("uplift", []))), lo, hi


def gather_gauges(t, e, lo: int, dist, n_total: int):
    """Gather per-rank gauge records (t: samples x local scenarios, e: samples x
    local scenarios x gauges) into whole-ensemble arrays on every rank,
    ordered by global scenario index.  All ranks record the same number of
    samples (one per coarse step)."""
    import numpy as np
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (lo, np.asarray(t), np.asarray(e)))
    parts.sort(key=lambda p: p[0])
    ts = [p[1] for p in parts if p[1].shape[1] > 0]
    es = [p[2] for p in parts if p[2].shape[1] > 0]
    T = np.concatenate(ts, axis=1)
    E = np.concatenate(es, axis=1)
    if T.shape[1] != n_total:
        raise RuntimeError("gathered scenario count does not match the ensemble")
    return T, E


def job_rate(units: float, seconds: float, dist=None) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (each rank passes its own units and its own elapsed time)."""
    if dist is None:
        return units / seconds
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64)
    s = torch.tensor([float(seconds)], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(s.item())
