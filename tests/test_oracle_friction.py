"""Pins of the oracle's Manning friction step (the drag D of Sec. 2.1, read
as D = g n^2 |u| / h^(4/3); the implicit step divides the momenta by
1 + dt D).

* uniform flow over a flat bed: the waves vanish, so only friction acts, and
  the momentum must equal the exact solution of
  d|m|/dt = -g n^2 |m|^2 / h^(7/3), |m|(t) = |m0| / (1 + g n^2 |m0| t / h^(7/3))
  (the implicit step is exact for this decay); two depths pin the exponent;
* friction acts along the flow: hv / hu stays exactly constant;
* n = 0 is the friction-free update bit for bit; still water with dry land
  stays exactly at rest.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

G = 9.81


def _uniform(h, u, v, n, dt, T):
    cfg = W.base_config(nx=6, ny=5, dx=100.0, dy=100.0, bc=[W.BC_EXTRAP] * 4, dt_max=dt, manning_n=n)
    L, M = cfg["nx"] * 100.0, cfg["ny"] * 100.0
    w = dict(cfg=cfg, topo=W.flat_topo(cfg, h), eta=[], uplift=[], gauges=np.zeros((0, 2)),
             uv=[(0, np.full((2, 2), u), np.full((2, 2), v), 0.0, 0.0, L, M)])
    o = W.load(oracle.Oracle(cfg), w)
    k = int(round(T / dt))
    o.step(k)
    hu, hv = o.level_array(0, 1, "hu"), o.level_array(0, 1, "hv")
    assert np.all(hu == hu[0, 0]) and np.all(hv == hv[0, 0])
    assert np.all(o.level_array(0, 1, "h") == h)
    return hu[0, 0], hv[0, 0], k * dt


def _exact(h, u, v, n, t):
    m0 = h * np.hypot(u, v)
    return m0 / (1.0 + G * n * n * m0 * t / h ** (7.0 / 3.0))


@pytest.mark.parametrize("h", [2.0, 8.0])
def test_uniform_flow_decay_matches_exact_solution(h):
    """For uniform flow the step is exact: 1 / |m| grows by g n^2 dt / h^(7/3)
    per step, which is the exact solution of d|m|/dt = -c |m|^2 sampled at
    the step times, whatever dt is."""
    u, v, n, T = 1.0, 0.5, 0.025, 600.0
    m0 = h * np.hypot(u, v)
    for dt in (2.0, 0.5):
        hu, hv, t = _uniform(h, u, v, n, dt, T)
        assert np.hypot(hu, hv) == pytest.approx(_exact(h, u, v, n, t), rel=1e-12)
        assert hv / hu == pytest.approx(v / u, rel=1e-14)
    assert 1.0 - _exact(h, u, v, n, T) / m0 > 0.01   # friction did something measurable


def test_zero_coefficient_is_the_friction_free_update():
    w = W.hump200()
    a = W.load(oracle.Oracle(w["cfg"]), w)
    cfg = dict(w["cfg"], manning_n=0.0)
    b = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
    a.step(20)
    b.step(20)
    for f in ("h", "hu", "hv"):
        assert np.array_equal(a.level_array(0, 1, f), b.level_array(0, 1, f))


def test_still_water_with_dry_land_stays_at_rest():
    w = W.lake_at_rest_shelf(n=64)
    cfg = dict(w["cfg"], manning_n=0.025)
    o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
    o.step(50)
    for f in ("hu", "hv"):
        assert np.abs(o.level_array(0, 1, f)).max() == 0.0


def test_friction_damps_a_hump_and_keeps_mass():
    w = W.hump200()
    cfg = dict(w["cfg"], manning_n=0.05)
    a = W.load(oracle.Oracle(w["cfg"]), w)
    b = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
    m0 = b.stats()["mass"]
    a.step(100)
    b.step(100)
    assert abs(b.stats()["mass"] - m0) <= 1e-13 * m0
    ka = np.sum(a.level_array(0, 1, "hu") ** 2 + a.level_array(0, 1, "hv") ** 2)
    kb = np.sum(b.level_array(0, 1, "hu") ** 2 + b.level_array(0, 1, "hv") ** 2)
    assert kb < ka
