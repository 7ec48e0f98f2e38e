"""Several GPUs, one process each: sharding of independent scenarios and the
whole-job throughput rule.

An ensemble's scenarios share nothing but the bathymetry: each advances with
its own time step, patches and gauges.  So they partition across ranks with no
collective on the data path.  Rank r builds its own context holding scenarios
[lo, hi), steps it, and only the finished gauge records are gathered at the
end.  A uniform single-scenario grid does not partition this way (that would
need halo exchange every level step); the benchmark runs a replica per rank.
The second half of the module is the host side of that exchange: a partition
of one level's patches over ranks and the schedule of its ghost halos.

Everything here is host logic over ``torch.distributed`` (any backend); the
solver is whatever object the caller passes (the CUDA binding where a GPU is present).
"""
from __future__ import annotations

import numpy as np


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


# ---------------------------------------------------------------------------
# Within one scenario: patches of a level spread over ranks.
#
# A level's patches are independent given their ghost cells (Sec. 3.1), so a
# scenario too large for one GPU splits by patches: each rank owns a set of
# patches, keeps them compact along a space-filling curve, and before every
# level step receives the 2-cell halos of its patches that other ranks own.
# Per level step the exchange is those halos (point to point) plus one
# all-reduce of the max wave speed; at a regrid the ranks all-gather the new
# patch lists.  These functions are the host side: the partition, the halo
# schedule, and a CPU data path over torch.distributed for the tests.  (No
# run here has more than one GPU, so the device data path -- ghost strips sent
# between the ghost fill and the update -- is not wired.)

def morton(i: int, j: int, bits: int = 16) -> int:
    """Z-order index of (i, j): the bits of i and j interleaved (i in the even bits)."""
    z = 0
    for b in range(bits):
        z |= ((i >> b) & 1) << (2 * b) | ((j >> b) & 1) << (2 * b + 1)
    return z


def partition_patches(boxes, world: int) -> list[int]:
    """Owner rank of each patch (boxes: (i0, j0, nx, ny) in level indices).
    Patches are ordered along the Z curve of their centres and the ordered
    list is cut into `world` contiguous runs of about equal cell count (a cut
    falls after the patch that takes the running total past k/world of it)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(boxes)
    order = sorted(range(n), key=lambda k: (morton(boxes[k][0] + boxes[k][2] // 2, boxes[k][1] + boxes[k][3] // 2), k))
    total = sum(b[2] * b[3] for b in boxes)
    owner = [0] * n
    acc, r = 0, 0
    for k in order:
        owner[k] = r
        acc += boxes[k][2] * boxes[k][3]
        while r + 1 < world and acc * world >= (r + 1) * total:
            r += 1
    return owner


def halo_schedule(boxes, owner, nxl: int, nyl: int, ghost: int = 2):
    """Messages of one level's halo exchange: a list of (src, dst, q, p, box)
    where rank src owns patch q, rank dst owns patch p, and box = (i0, j0, i1,
    j1), half-open in level indices, is the part of q's interior inside p's
    ghost ring (corners included) and inside the domain.  Pairs on the same
    rank need no message and are left out; the list is sorted (src, dst, q, p)
    so both sides walk it in the same order."""
    msgs = []
    for p, (pi, pj, pw, ph) in enumerate(boxes):
        gi0, gj0 = max(pi - ghost, 0), max(pj - ghost, 0)
        gi1, gj1 = min(pi + pw + ghost, nxl), min(pj + ph + ghost, nyl)
        for q, (qi, qj, qw, qh) in enumerate(boxes):
            if q == p or owner[q] == owner[p]:
                continue
            i0, j0 = max(gi0, qi), max(gj0, qj)
            i1, j1 = min(gi1, qi + qw), min(gj1, qj + qh)
            if i0 < i1 and j0 < j1:
                msgs.append((owner[q], owner[p], q, p, (i0, j0, i1, j1)))
    msgs.sort(key=lambda m: (m[0], m[1], m[2], m[3]))
    return msgs


def exchange_halos(fields: dict, boxes, owner, schedule, rank: int, dist, ghost: int = 2):
    """CPU data path of one halo exchange: `fields` maps each patch this rank
    owns to its (ny + 2 ghost, nx + 2 ghost) array (ghost ring included);
    for every message with this rank as source the interior block is sent, and
    every message with this rank as destination lands in the patch's ghost
    ring.  Sends and receives are posted together and then waited on."""
    import torch
    reqs, recv = [], []
    for (src, dst, q, p, (i0, j0, i1, j1)) in schedule:
        if src == rank:
            qi, qj = boxes[q][0], boxes[q][1]
            blk = fields[q][j0 - qj + ghost:j1 - qj + ghost, i0 - qi + ghost:i1 - qi + ghost]
            reqs.append(dist.isend(torch.from_numpy(blk.copy()), dst))
        elif dst == rank:
            buf = torch.empty((j1 - j0, i1 - i0), dtype=torch.float64)
            reqs.append(dist.irecv(buf, src))
            recv.append((p, (i0, j0, i1, j1), buf))
    for r in reqs:
        r.wait()
    for p, (i0, j0, i1, j1), buf in recv:
        pi, pj = boxes[p][0], boxes[p][1]
        fields[p][j0 - pj + ghost:j1 - pj + ghost, i0 - pi + ghost:i1 - pi + ghost] = buf.numpy()


def max_speed(local: float, dist) -> float:
    """The level's max wave speed over all ranks (the one collective of a level step)."""
    import torch
    t = torch.tensor([local], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allgather_flags(local_flags, dist):
    """The level's flag mask at a regrid, from the masks of all ranks.

    Each rank flags only the cells of the patches it owns, so a rank's mask is
    the level's full (ny, nx) extent with its own flags set.  The ranks send
    their flagged cells as sorted linear indices (a regrid flags a small part of
    a level) and every rank gets the union.  The clustering that follows is
    deterministic, so every rank then derives the same patch list and, through
    `partition_patches`, the same owners: no patch list is exchanged."""
    import torch
    mask = np.asarray(local_flags)
    mine = torch.from_numpy(np.flatnonzero(mask).astype(np.int64))
    n = torch.tensor([mine.numel()], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(dist.get_world_size())]
    dist.all_gather(counts, n)
    top = max(int(c.item()) for c in counts)
    pad = torch.full((top,), -1, dtype=torch.int64)
    pad[:mine.numel()] = mine
    parts = [torch.empty(top, dtype=torch.int64) for _ in counts]
    dist.all_gather(parts, pad)
    out = np.zeros(mask.size, dtype=np.uint8)
    for c, p in zip(counts, parts):
        out[p[:int(c.item())].numpy()] = 1
    return out.reshape(mask.shape)


def halo_messages(schedule, rank: int):
    """One rank's side of a halo exchange as message tables for the library's
    tsu_halo_pack / tsu_halo_unpack: ``send`` rows (q, i0, j0, i1, j1) of the
    messages this rank sources, ``recv`` rows (p, i0, j0, i1, j1) of those it
    receives, both in schedule order (sorted by peer), and for each the element
    range [lo, hi) of every peer's part of the buffer (3 fields per cell:
    q0, hu, hv)."""
    def side(rows):
        table, ranges, off = [], {}, 0
        for peer, k, box in rows:
            n = 3 * (box[2] - box[0]) * (box[3] - box[1])
            lo, _ = ranges.get(peer, (off, off))
            ranges[peer] = (lo, off + n)
            table.append((k, *box))
            off += n
        return np.array(table, dtype=np.int32).reshape(-1, 5), ranges, off
    send = side([(dst, q, box) for (src, dst, q, p, box) in schedule if src == rank])
    recv = side([(src, p, box) for (src, dst, q, p, box) in schedule if dst == rank])
    return send, recv


def exchange_halos_device(solver, scen: int, level: int, schedule, rank: int, dist, torch, device, dtype):
    """Device data path of one halo exchange: the boxes this rank sources are
    packed from its patches into one buffer on ``device`` (solver.halo_pack),
    each peer's slice is sent and the incoming slices received in one batch of
    point-to-point operations (NCCL between GPUs), and the received boxes are
    unpacked into the ghost rings (solver.halo_unpack).  ``solver`` is the
    library context (tsu_halo_pack / tsu_halo_unpack take device pointers) or
    any object with the same two methods."""
    (stab, sranges, sn), (rtab, rranges, rn) = halo_messages(schedule, rank)
    sbuf = torch.empty(max(sn, 1), dtype=dtype, device=device)
    rbuf = torch.empty(max(rn, 1), dtype=dtype, device=device)
    if len(stab):
        solver.halo_pack(scen, level, stab, sbuf.data_ptr(), sn)
    ops = [dist.P2POp(dist.isend, sbuf[lo:hi], peer) for peer, (lo, hi) in sorted(sranges.items())]
    ops += [dist.P2POp(dist.irecv, rbuf[lo:hi], peer) for peer, (lo, hi) in sorted(rranges.items())]
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    if len(rtab):
        solver.halo_unpack(scen, level, rtab, rbuf.data_ptr(), rn)
