"""The N > 1 path on CPU: world-size-2 gloo ranks.

* scenario sharding covers every scenario exactly once;
* an ensemble advanced as two shards (one context per rank, no collective on
  the data path) and gathered at the end is bit for bit the single-context
  run (scenarios are independent: own dt, patches, gauges);
* the whole-job rate is the units of all ranks over the slowest rank's time;
* one level's patches split over ranks: the partition balances cells along
  the Z curve, the halo schedule covers each ghost cell once, and a level
  stepped as two ranks exchanging halos is bit for bit the whole level.

The per-rank solver here is the oracle; with a GPU the same host logic
drives the CUDA binding.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1901_06798_gb300 import ranks
from paper_1901_06798_gb300 import workloads as W


def test_shard_covers_each_unit_once():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                lo, hi = ranks.shard(n, r, world)
                got += list(range(lo, hi))
                assert hi - lo in (n // world, n // world + 1)
            assert got == list(range(n))
    with pytest.raises(ValueError):
        ranks.shard(4, 2, 2)


def _workload():
    w = W.ensemble(n_scen=5, n=32, dx=16000.0, steps=6, seed=11)
    return dict(w, cfg=dict(w["cfg"], regrid_interval=2))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        w = _workload()
        part, lo, hi = ranks.shard_workload(w, rank, world)
        o = W.load(oracle.Oracle(part["cfg"]), part)
        o.step(w["steps"])
        t, e = o.read_gauges()
        T, E = ranks.gather_gauges(t, e, lo, dist, w["cfg"]["n_scenarios"])
        rate = ranks.job_rate(10.0 * (rank + 1), 1.0 + rank, dist)
        if rank == 0:
            np.savez(os.path.join(out_dir, "sharded.npz"), T=T, E=E, rate=rate)
    finally:
        dist.destroy_process_group()


def test_two_rank_ensemble_equals_single_context(tmp_path):
    import oracle
    oracle.build("parity")
    world = 2
    mp.start_processes(_rank_main, args=(world, _port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "sharded.npz")
    w = _workload()
    o = W.load(oracle.Oracle(w["cfg"]), w)
    o.step(w["steps"])
    t, e = o.read_gauges()
    assert got["T"].shape == t.shape and got["E"].shape == e.shape
    assert np.array_equal(got["T"], t)
    assert np.array_equal(got["E"], e)
    # 10 + 20 units over max(1, 2) seconds
    assert float(got["rate"]) == 15.0


# ---------------------------------------------------------------------------
# Within one scenario: a level's patches spread over ranks, ghost halos
# exchanged point to point before each step.

def _tiles(nx, ny, t):
    return [(i, j, min(t, nx - i), min(t, ny - j)) for j in range(0, ny, t) for i in range(0, nx, t)]


def _random_boxes(rng, n=40):
    """Disjoint boxes scattered over a 256 x 256 level (a refined level's patches)."""
    taken = np.zeros((256, 256), bool)
    out = []
    while len(out) < n:
        w, h = (int(v) for v in rng.integers(4, 40, 2))
        i, j = (int(v) for v in rng.integers(0, 256 - 40, 2))
        if not taken[j:j + h, i:i + w].any():
            taken[j:j + h, i:i + w] = True
            out.append((i, j, w, h))
    return out


def test_morton_interleaves_bits():
    assert [ranks.morton(i, j) for j in range(2) for i in range(2)] == [0, 1, 2, 3]
    assert ranks.morton(2, 0) == 4 and ranks.morton(0, 2) == 8 and ranks.morton(3, 3) == 15
    assert ranks.morton(0xFFFF, 0) == 0x55555555 and ranks.morton(0, 0xFFFF) == 0xAAAAAAAA


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_partition_balances_cells(world):
    rng = np.random.default_rng(7)
    for boxes in (_tiles(200, 150, 16), _random_boxes(rng)):
        owner = ranks.partition_patches(boxes, world)
        assert len(owner) == len(boxes) and set(owner) <= set(range(world))
        cells = [b[2] * b[3] for b in boxes]
        load = np.bincount(owner, weights=cells, minlength=world)
        # a contiguous cut of the curve misses the even share by less than one patch
        assert np.abs(load - sum(cells) / world).max() <= max(cells)
        assert len(set(owner)) == min(world, len(boxes))
    assert ranks.partition_patches([], 4) == []
    with pytest.raises(ValueError):
        ranks.partition_patches(_tiles(8, 8, 4), 0)


def test_partition_follows_the_curve():
    """Owners are non-decreasing along the Z order: each rank holds one run of
    the curve, so its patches are compact and its halo short."""
    boxes = _tiles(256, 256, 16)
    owner = ranks.partition_patches(boxes, 4)
    order = sorted(range(len(boxes)), key=lambda k: ranks.morton(boxes[k][0] + 8, boxes[k][1] + 8))
    assert [owner[k] for k in order] == sorted(owner)
    # 16 x 16 tiles into 4 ranks: the Z curve gives each rank one quadrant
    for k, (i, j, _, _) in enumerate(boxes):
        assert owner[k] == (i >= 128) + 2 * (j >= 128)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_halo_schedule_covers_every_ghost_cell_once(world):
    nx, ny = 61, 47
    boxes = _tiles(nx, ny, 9)
    owner = ranks.partition_patches(boxes, world)
    msgs = ranks.halo_schedule(boxes, owner, nx, ny)
    assert msgs == sorted(msgs, key=lambda m: m[:4])
    cover = {p: np.zeros((h + 4, w + 4), int) for p, (_, _, w, h) in enumerate(boxes)}
    for src, dst, q, p, (i0, j0, i1, j1) in msgs:
        assert src == owner[q] and dst == owner[p] and src != dst
        qi, qj, qw, qh = boxes[q]
        assert qi <= i0 < i1 <= qi + qw and qj <= j0 < j1 <= qj + qh        # inside q's interior
        pi, pj = boxes[p][:2]
        cover[p][j0 - pj + 2:j1 - pj + 2, i0 - pi + 2:i1 - pi + 2] += 1
    for p, (pi, pj, pw, ph) in enumerate(boxes):
        # same-rank neighbours fill the rest of the ghost ring locally
        for q, (qi, qj, qw, qh) in enumerate(boxes):
            if q != p and owner[q] == owner[p]:
                i0, j0 = max(pi - 2, qi), max(pj - 2, qj)
                i1, j1 = min(pi + pw + 2, qi + qw), min(pj + ph + 2, qj + qh)
                if i0 < i1 and j0 < j1:
                    cover[p][j0 - pj + 2:j1 - pj + 2, i0 - pi + 2:i1 - pi + 2] += 1
        jj, ii = np.mgrid[pj - 2:pj + ph + 2, pi - 2:pi + pw + 2]
        inside = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny)
        interior = (ii >= pi) & (ii < pi + pw) & (jj >= pj) & (jj < pj + ph)
        ring = inside & ~interior
        assert (cover[p][ring] == 1).all(), p
        assert (cover[p][~ring] == 0).all(), p


def _level_state(nx, ny, dx):
    """A wet-dry level: a hump of water over a bottom with an island, moving."""
    y, x = np.mgrid[0:ny, 0:nx] * dx + dx / 2
    B = -10.0 + 13.0 * np.exp(-((x - 0.7 * nx * dx) ** 2 + (y - 0.35 * ny * dx) ** 2) / (0.08 * nx * dx) ** 2)
    eta = 0.8 * np.exp(-((x - 0.3 * nx * dx) ** 2 + (y - 0.55 * ny * dx) ** 2) / (0.12 * nx * dx) ** 2)
    h = np.maximum(eta - B, 0.0)
    hu = 0.4 * h * np.sin(x / (nx * dx) * 5.0)
    hv = -0.3 * h * np.cos(y / (ny * dx) * 4.0)
    return [h, hu, hv, B]


_G, _DRY, _DT, _DX = 9.81, 1e-3, 0.5, 10.0


def _whole_level_steps(state, steps):
    import oracle
    q = [a.copy() for a in state]
    for _ in range(steps):
        _, (h, hu, hv) = oracle.count_step_flops(*(np.pad(a, 2, mode="edge") for a in q), _G, _DRY, _DT, _DX, _DX)
        q[:3] = [a[2:-2, 2:-2] for a in (h, hu, hv)]
    return q


class _PadSolver:
    """Stands in for the library context on CPU ranks: halo_pack / halo_unpack
    over the ranks' padded patch arrays with the library's buffer layout (per
    message the fields q0, hu, hv, each a row-major box)."""

    def __init__(self, pad, boxes):
        self.pad, self.boxes = pad, boxes

    def _view(self, ptr, n):
        import ctypes
        return np.ctypeslib.as_array((ctypes.c_double * n).from_address(ptr))

    def _walk(self, msgs, ptr, n, unpack):
        buf, off = self._view(ptr, n), 0
        for k, i0, j0, i1, j1 in msgs:
            pi, pj = self.boxes[k][0], self.boxes[k][1]
            for f in range(3):
                a = self.pad[k][f]
                blk = (slice(j0 - pj + 2, j1 - pj + 2), slice(i0 - pi + 2, i1 - pi + 2))
                m = (i1 - i0) * (j1 - j0)
                if unpack:
                    a[blk] = buf[off:off + m].reshape(j1 - j0, i1 - i0)
                else:
                    buf[off:off + m] = a[blk].ravel()
                off += m

    def halo_pack(self, scen, level, msgs, ptr, n):
        self._walk(msgs, ptr, n, False)

    def halo_unpack(self, scen, level, msgs, ptr, n):
        self._walk(msgs, ptr, n, True)


def _level_rank_main(rank, world, port, out_dir, nx, ny, tile, steps, device_path=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        boxes = _tiles(nx, ny, tile)
        owner = ranks.partition_patches(boxes, world)
        msgs = ranks.halo_schedule(boxes, owner, nx, ny)
        state = _level_state(nx, ny, _DX)
        mine = [p for p in range(len(boxes)) if owner[p] == rank]
        # each rank holds only its patches: (ny + 4, nx + 4) per field, ghosts included
        pad = {p: [np.zeros((boxes[p][3] + 4, boxes[p][2] + 4)) for _ in range(4)] for p in mine}
        for p in mine:
            i, j, w, h = boxes[p]
            for f in range(4):
                pad[p][f][2:-2, 2:-2] = state[f][j:j + h, i:i + w]
        sent = 0
        if device_path:   # B once; the state every step through the packed-buffer path
            ranks.exchange_halos({p: pad[p][3] for p in mine}, boxes, owner, msgs, rank, dist)
        for _ in range(steps):
            if device_path:
                ranks.exchange_halos_device(_PadSolver(pad, boxes), 0, 1, msgs, rank, dist, torch, "cpu",
                                            torch.float64)
            for f in range(4):
                fields = {p: pad[p][f] for p in mine}
                if not device_path:
                    ranks.exchange_halos(fields, boxes, owner, msgs, rank, dist)
                for p in mine:                                    # same-rank neighbours
                    pi, pj, pw, ph = boxes[p]
                    for q in mine:
                        qi, qj, qw, qh = boxes[q]
                        i0, j0 = max(pi - 2, qi), max(pj - 2, qj)
                        i1, j1 = min(pi + pw + 2, qi + qw), min(pj + ph + 2, qj + qh)
                        if q != p and i0 < i1 and j0 < j1:
                            pad[p][f][j0 - pj + 2:j1 - pj + 2, i0 - pi + 2:i1 - pi + 2] = \
                                pad[q][f][j0 - qj + 2:j1 - qj + 2, i0 - qi + 2:i1 - qi + 2]
                for p in mine:                                    # extrapolation outside the domain
                    pi, pj, pw, ph = boxes[p]
                    jj = np.clip(np.arange(pj - 2, pj + ph + 2), 0, ny - 1) - pj + 2
                    ii = np.clip(np.arange(pi - 2, pi + pw + 2), 0, nx - 1) - pi + 2
                    pad[p][f] = pad[p][f][np.ix_(jj, ii)]
            sent += sum((m[4][2] - m[4][0]) * (m[4][3] - m[4][1]) for m in msgs if m[0] == rank)
            for p in mine:
                _, new = oracle.count_step_flops(*pad[p], _G, _DRY, _DT, _DX, _DX)
                for f in range(3):
                    pad[p][f][2:-2, 2:-2] = new[f][2:-2, 2:-2]
        smax = max(float(np.abs(pad[p][1][2:-2, 2:-2]).max()) for p in mine)
        gmax = ranks.max_speed(smax, dist)
        out = [np.full((ny, nx), np.nan) for _ in range(3)]
        for p in mine:
            i, j, w, h = boxes[p]
            for f in range(3):
                out[f][j:j + h, i:i + w] = pad[p][f][2:-2, 2:-2]
        np.savez(os.path.join(out_dir, f"level_rank{rank}{'_dev' if device_path else ''}.npz"), h=out[0], hu=out[1],
                 hv=out[2], smax=smax, gmax=gmax, sent=sent)
    finally:
        dist.destroy_process_group()


def test_two_rank_level_step_equals_whole_level(tmp_path):
    """A 61 x 47 level in 9 x 9 patches (ragged last row and column), split over
    two ranks: after four steps with the halos exchanged each step, the union
    of the ranks' patches is bit for bit four oracle steps of the whole level."""
    import oracle
    oracle.build_flopcount()
    nx, ny, tile, steps, world = 61, 47, 9, 4, 2
    mp.start_processes(_level_rank_main, args=(world, _port(), str(tmp_path), nx, ny, tile, steps),
                       nprocs=world, join=True, start_method="spawn")
    parts = [np.load(tmp_path / f"level_rank{r}.npz") for r in range(world)]
    ref = _whole_level_steps(_level_state(nx, ny, _DX), steps)
    assert (ref[0] == 0.0).any() and (ref[0] > 0.0).any()            # wet and dry cells both present
    for k, f in enumerate(("h", "hu", "hv")):
        got = np.where(np.isnan(parts[0][f]), parts[1][f], parts[0][f])
        assert not np.isnan(got).any()
        assert np.isnan(parts[0][f]).sum() + np.isnan(parts[1][f]).sum() == nx * ny   # each cell on one rank
        assert np.array_equal(got, ref[k]), f
    # the all-reduce gives both ranks the larger of the two local maxima
    assert float(parts[0]["gmax"]) == float(parts[1]["gmax"]) == max(float(p["smax"]) for p in parts)
    # halo cells moved per step and field, against the level's cells
    boxes = _tiles(nx, ny, tile)
    owner = ranks.partition_patches(boxes, world)
    cut = sum((b[2] - b[0]) * (b[3] - b[1]) for *_, b in ranks.halo_schedule(boxes, owner, nx, ny))
    assert sum(int(p["sent"]) for p in parts) == cut * steps
    assert cut < 0.25 * nx * ny


def _regrid_rank_main(rank, world, port, out_dir):
    """Each rank flags |eta| > tol only inside the patches it owns; after the
    flag all-gather every rank clusters and partitions on its own."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        nx, ny = 96, 80
        boxes = _tiles(nx, ny, 16)
        owner = ranks.partition_patches(boxes, world)
        flags = _flags(nx, ny)
        local = np.zeros_like(flags)
        for p, (i, j, w, h) in enumerate(boxes):
            if owner[p] == rank:
                local[j:j + h, i:i + w] = flags[j:j + h, i:i + w]
        full = ranks.allgather_flags(local, dist)
        new = [tuple(int(v) for v in b) for b in oracle.cluster(full, eff=0.7)]
        np.savez(os.path.join(out_dir, f"regrid_rank{rank}.npz"), full=full, local=local,
                 boxes=np.array(new), owner=np.array(ranks.partition_patches(new, world)))
    finally:
        dist.destroy_process_group()


def _flags(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx]
    ring = np.abs(np.hypot(x - 40.0, y - 35.0) - 22.0) < 3.0
    return (ring | ((x > 80) & (y < 10))).astype(np.uint8)


def test_two_rank_regrid_agrees_on_patches_and_owners(tmp_path):
    import oracle
    oracle.build("parity")
    world = 2
    mp.start_processes(_regrid_rank_main, args=(world, _port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [np.load(tmp_path / f"regrid_rank{r}.npz") for r in range(world)]
    flags = _flags(96, 80)
    ref = np.array([tuple(int(v) for v in b) for b in oracle.cluster(flags, eff=0.7)])
    assert got[0]["local"].sum() > 0 and got[1]["local"].sum() > 0       # both ranks flagged something
    for g in got:
        assert np.array_equal(g["full"], flags)                          # the union is the whole mask
        assert np.array_equal(g["boxes"], ref)                           # the single-process patch list
    assert np.array_equal(got[0]["owner"], got[1]["owner"])
    assert set(got[0]["owner"].tolist()) == {0, 1}


def test_halo_messages_split_the_schedule_by_peer():
    boxes = _tiles(61, 47, 9)
    owner = ranks.partition_patches(boxes, 3)
    sched = ranks.halo_schedule(boxes, owner, 61, 47)
    for r in range(3):
        (st, sr, sn), (rt, rr, rn) = ranks.halo_messages(sched, r)
        mine_out = [m for m in sched if m[0] == r]
        mine_in = [m for m in sched if m[1] == r]
        assert [tuple(x) for x in st] == [(m[2], *m[4]) for m in mine_out]
        assert [tuple(x) for x in rt] == [(m[3], *m[4]) for m in mine_in]
        cells = lambda ms: 3 * sum((b[2] - b[0]) * (b[3] - b[1]) for *_, b in ms)
        assert sn == cells(mine_out) and rn == cells(mine_in)
        # each peer's slice holds exactly its messages, and the slices tile the buffer in peer order
        for rng, ms, peer_of in ((sr, mine_out, 1), (rr, mine_in, 0)):
            edges = sorted(rng.values())
            assert edges[0][0] == 0 and all(a[1] == b[0] for a, b in zip(edges, edges[1:]))
            for peer, (lo, hi) in rng.items():
                assert hi - lo == cells([m for m in ms if m[peer_of] == peer])


def test_two_rank_level_step_through_packed_buffers(tmp_path):
    """The same split level with the state's halos moved the way the device
    path moves them: each rank packs the boxes it sources into one buffer
    (tsu_halo_pack's layout), sends every peer its slice and receives its own
    in one batch of point-to-point operations, and unpacks them into the ghost
    rings.  Bit for bit the whole level after four steps."""
    import oracle
    oracle.build_flopcount()
    nx, ny, tile, steps, world = 61, 47, 9, 4, 2
    mp.start_processes(_level_rank_main, args=(world, _port(), str(tmp_path), nx, ny, tile, steps, True),
                       nprocs=world, join=True, start_method="spawn")
    parts = [np.load(tmp_path / f"level_rank{r}_dev.npz") for r in range(world)]
    ref = _whole_level_steps(_level_state(nx, ny, _DX), steps)
    for k, f in enumerate(("h", "hu", "hv")):
        got = np.where(np.isnan(parts[0][f]), parts[1][f], parts[0][f])
        assert np.array_equal(got, ref[k]), f

