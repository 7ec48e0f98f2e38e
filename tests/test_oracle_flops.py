"""Algorithmic operation counts of one cell update (the measurement's flop
count), from the oracle's patch update compiled with a counting scalar type
(oracle/flopcount.cpp: swe.c unchanged, `double` counting every operation).

Pins: the counting build computes exactly what the oracle computes (same bits
as a one-level oracle step); the square roots of an all-wet patch follow the
closed form 5 per Riemann problem (sqrt(g h) and sqrt(h) of both cells and the
Roe celerity) times the number of problems of the two sweeps.  The counts per
cell are printed with -s.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W


def _padded(o, f):
    return np.pad(o.level_array(0, 1, f), 2, mode="edge")


def _hump(nx=60, ny=50, dt=0.4):
    cfg = W.base_config(nx=nx, ny=ny, dx=10.0, dy=10.0, bc=[W.BC_EXTRAP] * 4, dt_max=dt)
    eta = W.gaussian_grid(0.0, 0.0, nx * 10.0, ny * 10.0, nx + 1, ny + 1, 310.0, 240.0, 0.5, 80.0, 60.0)
    return dict(cfg=cfg, topo=W.flat_topo(cfg, 10.0), eta=[(0, *eta)], uplift=[], gauges=np.zeros((0, 2)))


def test_counting_build_is_the_oracle_step():
    w = _hump()
    o = W.load(oracle.Oracle(w["cfg"]), w)
    h, hu, hv, B = (_padded(o, f) for f in ("h", "hu", "hv", "B"))
    o.step(1)
    assert o.stats()["dt"] == 0.4
    _, (h1, hu1, hv1) = oracle.count_step_flops(h, hu, hv, B, 9.81, 1e-3, 0.4, 10.0, 10.0)
    for mine, f in ((h1, "h"), (hu1, "hu"), (hv1, "hv")):
        assert np.array_equal(mine[2:-2, 2:-2], o.level_array(0, 1, f)), f


def test_sqrt_count_closed_form_all_wet():
    nx, ny = 60, 50
    w = _hump(nx, ny)
    o = W.load(oracle.Oracle(w["cfg"]), w)
    c, _ = oracle.count_step_flops(*(_padded(o, f) for f in ("h", "hu", "hv", "B")), 9.81, 1e-3, 0.4, 10.0, 10.0)
    # x sweep: ny + 4 rows of nx + 3 problems; y sweep: nx columns of ny + 3
    assert c["sqrt"] == 5 * ((ny + 4) * (nx + 3) + nx * (ny + 3))


@pytest.mark.parametrize("name", ["hump200", "shelf192"])
def test_counts_per_cell_update(name):
    if name == "hump200":
        w = W.hump200()
        n, dt, dx = 200, 0.5, 10.0
    else:
        w = W.shelf(n=192, dx=2000.0)
        n, dt, dx = 192, 5.0, 2000.0
    o = W.load(oracle.Oracle(w["cfg"]), w)
    o.step(10)
    dry = float((o.level_array(0, 1, "h") < 1e-3).mean())
    c, _ = oracle.count_step_flops(*(_padded(o, f) for f in ("h", "hu", "hv", "B")), 9.81, 1e-3, dt, dx, dx)
    per = {k: v / (n * n) for k, v in c.items()}
    flops = per["add"] + per["mul"] + per["div"] + per["sqrt"]
    print(f"\n{name}: dry {dry:.3f}; per cell update: " + ", ".join(f"{k} {v:.2f}" for k, v in per.items())
          + f"; flops (add+mul+div+sqrt) {flops:.1f}")
    # two sweeps of about one Riemann problem per cell, five square roots each
    assert 9.5 < per["sqrt"] < 10.6
    assert 200.0 < flops < 500.0
