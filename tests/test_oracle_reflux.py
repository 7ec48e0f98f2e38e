"""Refluxing (Sec. 3.1 step 5, which the paper drops on the GPU), as an option
of the FP64 oracle, for the study the paper's claim invites: how much does it
change a tsunami run?

Pins: with refluxing the mass of a closed flat basin is conserved to rounding
under 2- and 3-level AMR, while without it drifts by the flux mismatch at the
coarse-fine edges (so the pin measures the correction, not an accident); still
water over the shelf stays still.  The study (printed with -s) runs the
3-level shelf with the uplift and the coast, with and without refluxing, and
reports the gauge and mass differences.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W


def _basin(reflux, levels, steps=60):
    n, dx = 48, 100.0
    ratios = [4] if levels == 2 else [2, 4]
    cfg = W.base_config(nx=n, ny=n, dx=dx, dy=dx, bc=[W.BC_WALL] * 4, num_levels=levels, ratios=ratios,
                        regrid_interval=4, regions=[[1200.0, 1200.0, 3600.0, 3600.0, levels, levels]],
                        reflux=reflux)
    eta = W.gaussian_grid(0, 0, n * dx, n * dx, n + 1, n + 1, 1500.0, 2400.0, 0.5, 300.0, 300.0)
    w = dict(cfg=cfg, topo=W.flat_topo(cfg, 10.0), eta=[(0, *eta)], uplift=[],
             gauges=np.array([[2400.0, 2400.0], [600.0, 600.0]]))
    o = W.load(oracle.Oracle(cfg), w)
    m0 = o.stats()["mass"]
    o.step(steps)
    st = o.stats()
    assert st["cfl_violations"] == 0
    assert st["patches"][levels - 1] > 0
    return (st["mass"] - m0) / m0, o.read_gauges()[1]


@pytest.mark.parametrize("levels", [2, 3])
def test_reflux_conserves_mass_under_amr(levels):
    drift_on, e_on = _basin(1, levels)
    drift_off, e_off = _basin(0, levels)
    assert abs(drift_on) <= 1e-13
    assert abs(drift_off) > 1e-8          # the mismatch refluxing removes
    assert np.abs(e_on - e_off).max() > 0.0


def test_reflux_keeps_still_water_still():
    w = W.lake_at_rest_shelf(n=48)
    cfg = dict(w["cfg"], num_levels=2, ratios=[4], regrid_interval=4, flag_depth_below=200.0, reflux=1)
    o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
    o.step(20)
    assert o.num_patches(0, 2) > 0
    for lev in (1, 2):
        for f in ("hu", "hv"):
            a = o.level_array(0, lev, f)
            assert np.nanmax(np.abs(a)) == 0.0, (lev, f)


def test_reflux_rejects_unsplit_and_sphere():
    for extra in (dict(transverse=1), dict(spherical=1, x0=0.0, y0=10.0)):
        cfg = W.base_config(nx=10, ny=10, dx=1.0, dy=1.0, reflux=1, **extra)
        with pytest.raises(ValueError):
            oracle.Oracle(cfg)


def test_reflux_effect_on_the_shelf_tsunami():
    """The 3-level shelf (240 km, uplift, beach and dry land): gauges with and
    without refluxing after 16 coarse steps."""
    w = W.amr3(L=240e3, dx1=4000.0, steps=16)
    res = {}
    for rf in (0, 1):
        cfg = dict(w["cfg"], reflux=rf)
        o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
        m0 = o.stats()["mass"]
        o.step(16)
        _, e = o.read_gauges()
        res[rf] = (e, (o.stats()["mass"] - m0) / m0, o.stats()["patches"])
    e0, e1 = res[0][0], res[1][0]
    amp = np.abs(e0).max()
    diff = np.abs(e1 - e0).max()
    print(f"\nshelf 3-level, 16 coarse steps: max |eta| at gauges {amp:.4f} m, max gauge difference with "
          f"refluxing {diff:.3e} m ({diff / amp:.2e} of the amplitude); mass change without {res[0][1]:.2e}, "
          f"with {res[1][1]:.2e}; patches {res[0][2]} / {res[1][2]}")
    assert amp > 0.1
    assert diff < 0.05 * amp
