"""Checkpoint and restart through the C ABI: a run restored from a
checkpoint continues bit for bit like the run that wrote it -- every patch
of every level and scenario, the time, the gauge records and the counters --
in both precisions, across regrids (3-level AMR) and for an ensemble."""
import numpy as np
import pytest

from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _state(g, nlev, nscen):
    out = {}
    for s in range(nscen):
        for lev in range(1, nlev + 1):
            for box, a in g.patches(s, lev):
                for f in ("h", "hu", "hv", "B"):
                    out[(s, lev, tuple(int(v) for v in box), f)] = a[f]
    return out


@pytest.mark.parametrize("name,precision", [("amr", 0), ("amr", 1), ("ensemble", 1)])
def test_restart_continues_bit_for_bit(name, precision):
    from paper_1901_06798_gb300 import binding
    if name == "amr":
        w = W.amr3(L=240e3, dx1=4000.0, steps=6)
        w = dict(w, cfg=dict(w["cfg"], regrid_interval=2))
    else:
        w = W.ensemble(n_scen=3, n=64, dx=8000.0, steps=6)
    cfg = w["cfg"]
    nlev, nscen = cfg["num_levels"], cfg["n_scenarios"]
    a = W.load(binding.Tsunami(cfg, precision=precision), w)
    a.step(5)
    ck = a.checkpoint()
    a.step(7)
    b = W.load(binding.Tsunami(cfg, precision=precision), w)
    b.step(1)                 # a different history: the restore replaces all of it
    b.restore(ck)
    b.step(7)
    sa, sb = _state(a, nlev, nscen), _state(b, nlev, nscen)
    assert sa.keys() == sb.keys()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    ta, ea = a.read_gauges()
    tb, eb = b.read_gauges()
    assert np.array_equal(ta, tb) and np.array_equal(ea, eb)
    for s in range(nscen):
        xa, xb = a.stats(s), b.stats(s)
        for k in ("t", "dt", "cell_updates", "cfl_violations"):
            assert xa[k] == xb[k], (s, k)
        assert xa["patches"] == xb["patches"]


def test_restore_rejects_another_configuration():
    from paper_1901_06798_gb300 import binding
    w = W.hump200()
    a = W.load(binding.Tsunami(w["cfg"], precision=0), w)
    a.step(2)
    ck = a.checkpoint()
    cfg = dict(w["cfg"], dx=11.0, dy=11.0)
    b = W.load(binding.Tsunami(cfg, precision=0), dict(w, cfg=cfg))
    with pytest.raises(binding.TsuError):
        b.restore(ck)
    with pytest.raises(binding.TsuError):
        b.restore(ck[: len(ck) // 2])
    c = W.load(binding.Tsunami(w["cfg"], precision=0), w)
    with pytest.raises(binding.TsuError):
        c.restore(ck[: len(ck) // 2])   # truncated
    c.restore(ck)
    a.step(3)
    c.step(3)
    assert np.array_equal(a.level_array(0, 1, "h"), c.level_array(0, 1, "h"))
