"""GPU parity of the unsplit update with transverse corrections (the
original GeoClaw scheme that Sec. 5 compares the split GPU scheme against)
through the C ABI, against the FP64 oracle.

Bars: FP64 bit for bit (the kernel follows the oracle's operation order and
is built without contraction); FP32 perturbation form within 1e-4 m of
surface elevation.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F32P_ETA = 1e-4


def _pair(w, steps, precision=0, cfg=None, tuning=None):
    from paper_1901_06798_gb300 import binding
    cfg = dict(cfg or w["cfg"], transverse=1)
    w = dict(w, cfg=cfg)
    o = W.load(oracle.Oracle(cfg), w)
    g = binding.Tsunami(cfg, precision=precision)
    if tuning:
        g.set_tuning(*tuning)
    W.load(g, w)
    o.step(steps)
    g.step(steps)
    return o, g


def _bitwise(o, g, nlev=1):
    for lev in range(1, nlev + 1):
        ob = [p[0] for p in o.patches(0, lev)]
        gb = [tuple(int(v) for v in b) for b in g.boxes(0, lev)]
        assert ob == gb, lev
        for (box, a), (_, b) in zip(o.patches(0, lev), g.patches(0, lev)):
            for f in ("h", "hu", "hv"):
                assert np.array_equal(a[f], b[f]), (lev, box, f, np.abs(a[f] - b[f]).max())


def test_hump_f64_bitwise():
    o, g = _pair(W.hump200(), 100)
    _bitwise(o, g)
    so, sg = o.stats(), g.stats()
    assert so["dt"] == sg["dt"] and so["t"] == sg["t"]


@pytest.mark.parametrize("tuning", [(64, 32), (128, 64), (256, 128), (64, 7)])
def test_launch_shapes_and_ragged_strips_bitwise(tuning):
    w = W.hump200()
    cfg = dict(w["cfg"], nx=133, ny=71)
    o, g = _pair(dict(w, cfg=cfg), 25, cfg=cfg, tuning=tuning)
    _bitwise(o, g)


def test_tiles_and_anisotropic_cells_bitwise():
    w = W.hump200()
    cfg = dict(w["cfg"], level1_tile=37)
    o, g = _pair(w, 30, cfg=cfg)
    assert g.num_patches(0, 1) == 36
    _bitwise(o, g)
    cfg = dict(w["cfg"], ny=100, dy=20.0, bc=[W.BC_EXTRAP, W.BC_WALL, W.BC_EXTRAP, W.BC_WALL])
    o, g = _pair(dict(w, cfg=cfg), 40, cfg=cfg)
    _bitwise(o, g)


def test_tiny_grid_bitwise():
    w = W.hump200()
    cfg = dict(w["cfg"], nx=5, ny=3, dx=400.0, dy=400.0, level1_tile=2)
    o, g = _pair(dict(w, cfg=cfg), 10, cfg=cfg)
    _bitwise(o, g)


def test_shelf_with_dry_land_f64_bitwise():
    w = W.shelf(n=192, dx=2000.0, steps=60)
    o, g = _pair(w, 60)
    _bitwise(o, g)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(eo, eg)


def test_amr3_f64_bitwise():
    w = W.amr3(L=240e3, dx1=4000.0, steps=6)
    o, g = _pair(w, 6)
    assert o.num_patches(0, 3) > 0
    _bitwise(o, g, 3)
    assert o.stats()["cell_updates"] == g.stats()["cell_updates"]


@pytest.mark.parametrize("name", ["hump", "shelf"])
def test_f32_perturbation_within_1e4_m(name):
    w = W.hump200() if name == "hump" else W.shelf(n=192, dx=2000.0, steps=100)
    o, g = _pair(w, 100, precision=1)
    wet = o.level_array(0, 1, "h") > 0
    assert np.abs(g.level_array(0, 1, "eta") - o.level_array(0, 1, "eta"))[wet].max() <= F32P_ETA
    _, eo = o.read_gauges()
    _, eg = g.read_gauges()
    assert np.abs(eg - eo).max() <= F32P_ETA


def test_f32_launch_shapes_agree_and_match_oracle():
    """FP32 on ragged strips: every launch shape gives the same bits (the shape
    only moves work between CTAs) and stays within the surface bar; also with
    2:1 cells and walls on two sides."""
    from paper_1901_06798_gb300 import binding
    w = W.hump200()
    for cfg, steps in ((dict(w["cfg"], nx=133, ny=71), 25),
                       (dict(w["cfg"], ny=100, dy=20.0, bc=[W.BC_EXTRAP, W.BC_WALL, W.BC_EXTRAP, W.BC_WALL]), 40)):
        cfg = dict(cfg, transverse=1)
        o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
        o.step(steps)
        wet = o.level_array(0, 1, "h") > 0
        ref = None
        for tuning in [(64, 32), (128, 64), (256, 128), (64, 7)]:
            g = W.load(binding.Tsunami(cfg, precision=1), dict(w, cfg=cfg))
            g.set_tuning(*tuning)
            g.step(steps)
            got = {f: g.level_array(0, 1, f) for f in ("eta", "hu", "hv")}
            g.close()
            if ref is None:
                ref = got
                assert np.abs(got["eta"] - o.level_array(0, 1, "eta"))[wet].max() <= F32P_ETA
            else:
                for f in got:
                    assert np.array_equal(got[f], ref[f]), (tuning, f)


def test_lake_at_rest_both_precisions():
    from paper_1901_06798_gb300 import binding
    w = W.lake_at_rest_shelf(n=96)
    cfg = dict(w["cfg"], transverse=1)
    for prec in (0, 1):
        g = W.load(binding.Tsunami(cfg, precision=prec), dict(w, cfg=cfg))
        g.step(200)
        for f in ("hu", "hv"):
            assert np.abs(g.level_array(0, 1, f)).max() == 0.0


def test_full_size_shelf4096_window():
    """The 4096^2 run with transverse corrections: a window around the
    uplift equals the oracle run on a crop holding its domain of dependence."""
    from paper_1901_06798_gb300 import binding
    w = W.shelf(n=4096, dx=500.0)
    cfg = dict(w["cfg"], transverse=1)
    k, dx = 3, 500.0
    g = W.load(binding.Tsunami(cfg, precision=0), dict(w, cfg=cfg, gauges=np.zeros((0, 2))))
    g.step(k)
    xs = (2048e3 - 600e3) + (np.arange(-200, 200) + 0.5) * dx
    ys = 1024e3 + (np.arange(-300, 300) + 0.5) * dx
    eta = g.read_field(0, 1, "eta", len(xs), len(ys), xs[0], ys[0], dx, dx)
    ci0, cj0 = int(xs[0] / dx) - 4 * k - 8, int(ys[0] / dx) - 4 * k - 8
    cw, ch = len(xs) + 2 * (4 * k + 8), len(ys) + 2 * (4 * k + 8)
    ccfg = dict(cfg, nx=cw, ny=ch, x0=ci0 * dx, y0=cj0 * dx)
    o = W.load(oracle.Oracle(ccfg), dict(w, cfg=ccfg, gauges=np.zeros((0, 2))))
    o.step(k)
    assert o.stats()["dt"] == g.stats()["dt"]
    eo = o.read_field(0, 1, "eta", len(xs), len(ys), xs[0], ys[0], dx, dx)
    assert np.nanmax(np.abs(eta - eo)) <= 1e-12 * np.nanmax(np.abs(eo))
