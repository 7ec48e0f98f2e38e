"""GPU parity at the horizon of the bar: 100 steps (100 coarse steps under
AMR) against the FP64 oracle, through the C ABI.

Bars: FP64 relative error per field <= 1e-12 (the FP64 kernels follow the
oracle's operation order without contraction, so the fields are compared bit
for bit); FP32 perturbation form: surface elevation within 1e-4 m per field on
every level and per gauge.  Each oracle run is shared by the FP64 and the FP32
comparison (module-scoped fixtures); the longest takes about 100 s on one core.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F32P_ETA = 1e-4


def _gpu(cfg, precision=0):
    from paper_1901_06798_gb300 import binding
    return binding.Tsunami(cfg, precision=precision)


def _run(w, steps, precision=None):
    obj = oracle.Oracle(w["cfg"]) if precision is None else _gpu(w["cfg"], precision)
    W.load(obj, w)
    for _ in range(steps // 10):
        obj.step(10)
    if steps % 10:
        obj.step(steps % 10)
    return obj


def _levels_bitwise(o, g, nlev, nscen=1):
    for s in range(nscen):
        for lev in range(1, nlev + 1):
            ob = [p[0] for p in o.patches(s, lev)]
            gb = [tuple(int(v) for v in b) for b in g.boxes(s, lev)]
            assert ob == gb, (s, lev)
            for (box, a), (_, b) in zip(o.patches(s, lev), g.patches(s, lev)):
                for f in ("h", "hu", "hv"):
                    assert np.array_equal(a[f], b[f]), (s, lev, box, f, np.abs(a[f] - b[f]).max())


def _levels_eta(o, g, nlev, nscen=1):
    """Largest |eta_gpu - eta_oracle| over wet cells of every level (FP32 runs
    may regrid differently near the flag threshold: compare where both hold
    the same patch)."""
    worst = 0.0
    for s in range(nscen):
        for lev in range(1, nlev + 1):
            gp = {tuple(int(v) for v in b): a for b, a in g.patches(s, lev)}
            for box, a in o.patches(s, lev):
                b = gp.get(tuple(box))
                if b is None:
                    continue
                wet = a["h"] > 1e-3
                if wet.any():
                    eo = (a["h"] + a["B"])[wet]
                    eg = (b["h"] + b["B"])[wet]
                    worst = max(worst, float(np.abs(eg - eo).max()))
    return worst


def _window():
    """A 512^2 window of the 4096^2, dx = 500 m shelf workload: 444-700 km
    offshore (the continental slope and the 2 m uplift centred 600 km out),
    centred on mid-y, extrapolating boundaries at the window's edges."""
    w = W.shelf(n=4096, dx=500.0)
    n, dx = 512, 500.0
    cfg = dict(w["cfg"], nx=n, ny=n, x0=2048e3 - 700e3, y0=1024e3 - 128e3)
    g = np.array([[2048e3 - 600e3, 1024e3], [2048e3 - 520e3, 1024e3 + 40e3], [2048e3 - 460e3, 1024e3 - 90e3]])
    return dict(w, cfg=cfg, gauges=g)


@pytest.fixture(scope="module")
def window100():
    w = _window()
    return w, _run(w, 100)


def test_shelf_window_512_f64_100_steps(window100):
    w, o = window100
    g = _run(w, 100, 0)
    _levels_bitwise(o, g, 1)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(to, tg) and np.array_equal(eo, eg)


def test_shelf_window_512_f32_100_steps(window100):
    w, o = window100
    g = _run(w, 100, 1)
    err = _levels_eta(o, g, 1)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    print(f"\nwindow 512^2, 100 steps: FP32 surface error {err:.2e} m, gauges {np.abs(eg - eo).max():.2e} m")
    assert err <= F32P_ETA and np.abs(eg - eo).max() <= F32P_ETA
    np.testing.assert_allclose(tg, to, rtol=1e-5)


def test_shelf_with_dry_land_100_steps_both_precisions():
    """192^2 cells of 2 km over the whole profile: deep water, slope, shelf,
    beach and dry land, the uplift's wave reaching the shelf."""
    w = W.shelf(n=192, dx=2000.0, steps=100)
    o = _run(w, 100)
    _levels_bitwise(o, _run(w, 100, 0), 1)
    assert _levels_eta(o, _run(w, 100, 1), 1) <= F32P_ETA


@pytest.fixture(scope="module")
def amr3_100():
    """3-level AMR (ratios 4, 4) over the shelf on the reduced 200 km domain,
    level-1 dx 4 km, 100 coarse steps (1600 steps of level 3) with regrids."""
    w = W.amr3(L=200e3, dx1=4000.0)
    return w, _run(w, 100)


def test_amr3_f64_100_coarse_steps(amr3_100):
    w, o = amr3_100
    g = _run(w, 100, 0)
    assert o.num_patches(0, 3) > 0
    _levels_bitwise(o, g, 3)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(to, tg) and np.array_equal(eo, eg)
    so, sg = o.stats(), g.stats()
    assert so["cell_updates"] == sg["cell_updates"] and so["cfl_retakes"] == sg["cfl_retakes"]


def test_amr3_f32_every_level_100_coarse_steps(amr3_100):
    w, o = amr3_100
    g = _run(w, 100, 1)
    err = _levels_eta(o, g, 3)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    gerr = np.abs(eg - eo).max()
    print(f"\namr3 100 coarse steps: FP32 surface error on every level {err:.2e} m, gauges {gerr:.2e} m")
    assert err <= F32P_ETA and gerr <= F32P_ETA


@pytest.fixture(scope="module")
def ensemble8():
    """8 scenarios of the ensemble workload (seed 1901 draws their uplift
    centres and amplitudes), 128^2 cells of 8 km and a ratio-4 level each,
    40 coarse steps."""
    w = W.ensemble(n_scen=8, n=128, dx=8000.0)
    return w, _run(w, 40)


def test_ensemble8_f64_40_coarse_steps(ensemble8):
    w, o = ensemble8
    g = _run(w, 40, 0)
    _levels_bitwise(o, g, 2, nscen=8)
    assert np.array_equal(o.read_gauges()[1], g.read_gauges()[1])


def test_ensemble8_f32_gauges_per_scenario(ensemble8):
    w, o = ensemble8
    g = _run(w, 40, 1)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    per = np.abs(eg - eo).max(axis=(0, 2))   # per scenario
    print("\nensemble FP32 gauge error per scenario (m):", " ".join(f"{v:.1e}" for v in per))
    assert per.shape == (8,) and per.max() <= F32P_ETA
    assert _levels_eta(o, g, 2, nscen=8) <= F32P_ETA


def test_amr4_bay_f32_gauges_40_coarse_steps():
    """4 levels (ratios 4, 4, 8) down to dx1 / 128 around the bay on a reduced
    domain, 10 gauges (deep water, shelf, bay), 40 coarse steps: FP64 bit for
    bit, FP32 gauges within 1e-4 m."""
    w = W.amr4_bay(L=150e3, dx1=3000.0, radius=1500.0, box=4000.0)
    o = _run(w, 40)
    assert o.num_patches(0, 4) > 0
    _levels_bitwise(o, _run(w, 40, 0), 4)
    g = _run(w, 40, 1)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert eo.shape[2] == 10
    gerr = np.abs(eg - eo).max()
    print(f"\nbay 40 coarse steps: FP32 gauge error {gerr:.2e} m")
    assert gerr <= F32P_ETA
