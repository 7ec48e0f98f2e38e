"""The N > 1 path on CPU: world-size-2 gloo ranks.

* scenario sharding covers every scenario exactly once;
* an ensemble advanced as two shards (one context per rank, no collective on
  the data path) and gathered at the end is bit for bit the single-context
  run (scenarios are independent: own dt, patches, gauges);
* the whole-job rate is the units of all ranks over the slowest rank's time.

The per-rank solver here is the oracle; on a GPU machine the same host logic
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
