"""GPU parity of the latitude-longitude (capacity form) update, through the C
ABI, against the FP64 oracle.

Bars: FP64 relative error per field <= 1e-12, and bit for bit where the
library and the oracle build the same capacity tables from the same host sin
and cos (uniform grids and the AMR run alike); patch lists bit-exact.  FP32
perturbation form: surface elevation within 1e-4 m of the oracle on wet cells
and at every gauge.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64_REL = 1e-12
F32P_ETA = 1e-4


def _pair(w, steps, precision=0):
    from paper_1901_06798_gb300 import binding
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g = W.load(binding.Tsunami(w["cfg"], precision=precision), w)
    o.step(steps)
    g.step(steps)
    return o, g


def _rel(a, b):
    m = np.nanmax(np.abs(b))
    return np.nanmax(np.abs(a - b)) / (m if m > 0 else 1.0)


def _basin(lat0=40.0, n=48, box=2.0, frac=0.65, dt_max=10.0):
    """A hump running up a sloping beach between walls at 40 N (the oracle's
    mass pin), at a fixed dt below the CFL limit."""
    d = box / n
    x0, y0 = 200.0, lat0 - box / 2
    cfg = W.base_config(nx=n, ny=n, x0=x0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1, dt_max=dt_max)
    xs = np.linspace(x0, x0 + box, n + 1)
    ys = np.linspace(y0, y0 + box, n + 1)
    X, Y = np.meshgrid(xs, ys)
    B = -60.0 + 75.0 * (X - x0) / box + 10.0 * np.sin(3.0 * (Y - y0))
    eta = W.gaussian_grid(x0, y0, box, box, n + 1, n + 1, x0 + frac * box, lat0 + 0.2, 2.0, 0.15, 0.2)[0]
    return dict(cfg=cfg, topo=[(B, x0, y0, d, d)], eta=[(0, eta, x0, y0, d, d)], uplift=[],
                gauges=np.array([[x0 + 0.5 * box, lat0], [x0 + 0.9 * box, lat0 + 0.3]]))


def _equator_hump(n=40, box=4.0):
    """A hump centred on the equator over a flat 500 m bed, CFL-driven dt."""
    d = box / n
    cfg = W.base_config(nx=n, ny=n, x0=100.0, y0=-box / 2, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1)
    eta = W.gaussian_grid(100.0, -box / 2, box, box, n + 1, n + 1, 101.5, 0.0, 1.0, 0.3, 0.4)
    return dict(cfg=cfg, topo=[(np.full((2, 2), -500.0), 100.0, -box / 2, box, box)], eta=[(0, *eta)], uplift=[],
                gauges=np.zeros((0, 2)))


def test_basin_with_wetting_and_drying_bitwise():
    w = _basin()
    o, g = _pair(w, 200)
    assert g.stats()["cfl_violations"] == 0
    for f in ("h", "hu", "hv"):
        a, b = o.level_array(0, 1, f), g.level_array(0, 1, f)
        assert np.array_equal(a, b), (f, np.abs(a - b).max())
    assert abs(g.stats()["mass"] - o.stats()["mass"]) <= 1e-12 * o.stats()["mass"]


def test_equator_hump_f64_and_symmetry():
    o, g = _pair(_equator_hump(), 80)
    for f in ("h", "hu", "hv"):
        assert _rel(g.level_array(0, 1, f), o.level_array(0, 1, f)) <= F64_REL, f
    h = g.level_array(0, 1, "h")
    assert np.abs(h - h[::-1, :]).max() <= 1e-12 * h.max()
    assert g.stats()["t"] == o.stats()["t"]


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_strip_shapes_f64(threads):
    """Every FP64 launch shape of the capacity-form kernel, on a grid whose
    width leaves a ragged last strip."""
    from paper_1901_06798_gb300 import binding
    w = _basin(n=150, box=3.0)
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g = W.load(binding.Tsunami(w["cfg"], precision=0), w)
    g.set_tuning(step_threads=threads)
    o.step(30)
    g.step(30)
    for f in ("h", "hu", "hv"):
        assert np.array_equal(o.level_array(0, 1, f), g.level_array(0, 1, f)), (threads, f)


def _amr_lonlat():
    return W.lonlat(W.amr3(L=240e3, dx1=4000.0, steps=6), lon0=142.0, lat0=35.0)


def test_amr3_lonlat_f64_patch_lists_fields_gauges():
    w = _amr_lonlat()
    o, g = _pair(w, 6)
    assert o.num_patches(0, 3) > 0
    for lev in (1, 2, 3):
        ob = [p[0] for p in o.patches(0, lev)]
        gb = [tuple(int(v) for v in b) for b in g.boxes(0, lev)]
        assert ob == gb, lev
        for (box, a), (_, b) in zip(o.patches(0, lev), g.patches(0, lev)):
            for f in ("h", "hu", "hv", "B"):
                assert np.array_equal(a[f], b[f]), (lev, box, f, _rel(b[f], a[f]))
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(to, tg) and np.array_equal(eo, eg)
    so, sg = o.stats(), g.stats()
    assert so["cell_updates"] == sg["cell_updates"]
    assert abs(sg["mass"] - so["mass"]) <= 1e-12 * so["mass"]


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
def test_f32_perturbation_within_1e4_m(threads):
    from paper_1901_06798_gb300 import binding
    w = _basin()
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g = W.load(binding.Tsunami(w["cfg"], precision=1), w)
    g.set_tuning(step_threads=threads)
    o.step(200)
    g.step(200)
    wet = o.level_array(0, 1, "h") > 0
    assert np.abs(g.level_array(0, 1, "eta") - o.level_array(0, 1, "eta"))[wet].max() <= F32P_ETA
    _, eo = o.read_gauges()
    _, eg = g.read_gauges()
    assert np.abs(eg - eo).max() <= F32P_ETA


def test_amr3_lonlat_f32p_gauges_within_1e4_m():
    w = _amr_lonlat()
    o, g = _pair(w, 6, precision=1)
    _, eo = o.read_gauges()
    _, eg = g.read_gauges()
    assert np.abs(eg - eo).max() <= F32P_ETA


def test_lake_at_rest_lonlat_both_precisions():
    w = _basin()
    w = dict(w, eta=[])
    for prec in (0, 1):
        o, g = _pair(w, 40, precision=prec)
        for f in ("hu", "hv"):
            assert np.abs(g.level_array(0, 1, f)).max() == 0.0, (prec, f)
