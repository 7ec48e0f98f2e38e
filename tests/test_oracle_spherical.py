"""Pins of the oracle's latitude-longitude (spherical) mode: the split step in
capacity form (cell capacity = zone area over an equatorial cell's, latitude
edges weighted by cos of their latitude, the divergence term of the varying
edge length in the mass equation).

* local plane limit: a small patch of sphere at latitude phi0 is, to
  O(dphi tan phi0), the Cartesian grid with dx = R cos(phi0) dlambda and
  dy = R dphi -- exact at the equator, and the difference grows with
  latitude as the capacity varies across the patch;
* mass in spherical area is conserved between walls, with wetting and
  drying;
* a hump centred on the equator stays mirror-symmetric north-south;
* still water with dry land stays at rest; uniform zonal flow stays uniform;
* a fully refined level 2 is bitwise the uniform fine grid.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

R = 6371.0e3
D2R = np.pi / 180.0


def _plane_limit_diff(lat0, n=60, box=0.6, steps=40, depth=200.0):
    d = box / n
    x0, y0 = 150.0, lat0 - box / 2
    cfg_s = W.base_config(nx=n, ny=n, x0=x0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1, dt_max=2.0)
    dxc, dyc = R * np.cos(lat0 * D2R) * d * D2R, R * d * D2R
    cfg_c = W.base_config(nx=n, ny=n, dx=dxc, dy=dyc, bc=[W.BC_WALL] * 4, dt_max=2.0)
    I, J = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    eta = 0.5 * np.exp(-((I - n / 2) ** 2 + (J - n / 2) ** 2) / (2 * (n / 10) ** 2))
    ws = dict(cfg=cfg_s, topo=[(np.full((2, 2), -depth), x0, y0, box, box)],
              eta=[(0, eta, x0 + 0.5 * d, y0 + 0.5 * d, d, d)], uplift=[], gauges=np.zeros((0, 2)))
    wc = dict(cfg=cfg_c, topo=[(np.full((2, 2), -depth), 0.0, 0.0, n * dxc, n * dyc)],
              eta=[(0, eta, 0.5 * dxc, 0.5 * dyc, dxc, dyc)], uplift=[], gauges=np.zeros((0, 2)))
    a, b = W.load(oracle.Oracle(cfg_s), ws), W.load(oracle.Oracle(cfg_c), wc)
    a.step(steps)
    b.step(steps)
    ea, eb = a.level_array(0, 1, "eta"), b.level_array(0, 1, "eta")
    return np.abs(ea - eb).max() / np.abs(eb).max()


def test_local_plane_limit():
    d0, d30, d45, d60 = (_plane_limit_diff(lat) for lat in (0.0, 30.0, 45.0, 60.0))
    assert d0 < 1e-6
    assert d45 < 2e-3 and d60 < 5e-3
    assert d0 < d30 < d45 < d60          # grows with the capacity's variation across the patch


def _basin(lat0=40.0, n=48, box=2.0, frac=0.65, dt_max=1e9):
    d = box / n
    x0, y0 = 200.0, lat0 - box / 2
    cfg = W.base_config(nx=n, ny=n, x0=x0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1, dt_max=dt_max)
    xs = np.linspace(x0, x0 + box, n + 1)
    ys = np.linspace(y0, y0 + box, n + 1)
    X, Y = np.meshgrid(xs, ys)
    B = -60.0 + 75.0 * (X - x0) / box + 10.0 * np.sin(3.0 * (Y - y0))
    eta = W.gaussian_grid(x0, y0, box, box, n + 1, n + 1, x0 + frac * box, lat0 + 0.2, 2.0, 0.15, 0.2)[0]
    return cfg, dict(cfg=cfg, topo=[(B, x0, y0, d, d)], eta=[(0, eta, x0, y0, d, d)], uplift=[],
                     gauges=np.zeros((0, 2)))


def test_mass_conserved_between_walls_with_wetting_and_drying():
    """At a fixed dt below the CFL limit (no step may exceed it, since steps
    are not retaken), a hump running up a beach at 40 N."""
    cfg, w = _basin(dt_max=10.0)
    o = W.load(oracle.Oracle(cfg), w)
    m0 = o.stats()["mass"]
    wet0 = o.level_array(0, 1, "h") > 0
    o.step(200)
    h = o.level_array(0, 1, "h")
    assert ((h > 0) != wet0).sum() > 0 and (~(h > 0)).sum() > 0
    assert o.stats()["cfl_violations"] == 0
    assert abs(o.stats()["mass"] - m0) <= 1e-12 * m0


def test_equator_mirror_symmetry():
    n, box = 40, 4.0
    d = box / n
    cfg = W.base_config(nx=n, ny=n, x0=100.0, y0=-box / 2, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1)
    eta = W.gaussian_grid(100.0, -box / 2, box, box, n + 1, n + 1, 101.5, 0.0, 1.0, 0.3, 0.4)
    w = dict(cfg=cfg, topo=[(np.full((2, 2), -500.0), 100.0, -box / 2, box, box)], eta=[(0, *eta)], uplift=[],
             gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    o.step(80)
    h, hv = o.level_array(0, 1, "h"), o.level_array(0, 1, "hv")
    assert np.abs(h - h[::-1, :]).max() <= 1e-12 * h.max()
    assert np.abs(hv + hv[::-1, :]).max() <= 1e-11 * np.abs(hv).max()   # rounding of the row latitudes


def test_still_water_and_uniform_zonal_flow():
    cfg, w = _basin()
    w = dict(w, eta=[])
    o = W.load(oracle.Oracle(cfg), w)
    o.step(60)
    for f in ("hu", "hv"):
        assert np.abs(o.level_array(0, 1, f)).max() == 0.0
    n, d = 30, 0.1
    cfg = W.base_config(nx=n, ny=n, x0=10.0, y0=30.0, dx=d, dy=d, bc=[W.BC_EXTRAP] * 4, spherical=1)
    w = dict(cfg=cfg, topo=[(np.full((2, 2), -300.0), 10.0, 30.0, 3.0, 3.0)], eta=[], uplift=[],
             gauges=np.zeros((0, 2)), uv=[(0, np.full((2, 2), 2.0), np.zeros((2, 2)), 10.0, 30.0, 3.0, 3.0)])
    o = W.load(oracle.Oracle(cfg), w)
    o.step(40)
    assert np.all(o.level_array(0, 1, "hu") == 600.0) and np.all(o.level_array(0, 1, "h") == 300.0)


def test_full_refinement_equals_fine_grid():
    n, box, r = 12, 1.2, 4
    d = box / n
    x0, y0 = 130.0, 35.0
    base = W.base_config(nx=n, ny=n, x0=x0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1)
    topo = [(np.array([[-80.0, -20.0], [-80.0, -20.0]]), x0, y0, box, box)]
    up = W.gaussian_grid(x0, y0, box, box, 65, 65, x0 + 0.5, y0 + 0.6, 0.8, 0.1, 0.12)
    dt = 8.0
    amr = dict(base, num_levels=2, ratios=[r], regrid_interval=2, patch_max=24, dt_max=dt,
               regions=[[x0 - 1, y0 - 1, x0 + box + 1, y0 + box + 1, 2, 2]])
    fine = W.base_config(nx=n * r, ny=n * r, x0=x0, y0=y0, dx=d / r, dy=d / r, bc=[W.BC_WALL] * 4, spherical=1,
                         level1_tile=29, dt_max=dt / r)
    a, b = oracle.Oracle(amr), oracle.Oracle(fine)
    for o in (a, b):
        o.add_topo(*topo[0])
        o.init()
        o.add_uplift(0, *up)
    for _ in range(3):
        a.step(1)
        b.step(r)
    for f in ("h", "hu", "hv"):
        assert np.array_equal(a.level_array(0, 2, f), b.level_array(0, 1, f))


def test_spherical_rejects_poles_and_transverse():
    cfg = W.base_config(nx=10, ny=10, x0=0.0, y0=85.0, dx=1.0, dy=1.0, spherical=1)
    with pytest.raises(ValueError):
        oracle.Oracle(cfg)
    cfg = W.base_config(nx=10, ny=10, x0=0.0, y0=10.0, dx=1.0, dy=1.0, spherical=1, transverse=1)
    with pytest.raises(ValueError):
        oracle.Oracle(cfg)


def _kappa(y0, dy, J):
    """Capacity of row J: zone area over the area of an equatorial cell."""
    a, b = (y0 + J * dy) * D2R, (y0 + (J + 1) * dy) * D2R
    return (np.sin(b) - np.sin(a)) / (dy * D2R)


def test_capacity_weighted_averaging_conserves_mass():
    """Full refinement over a flat bed with no dry cells: the averaged level-1
    mass equals the level-2 mass in spherical measure (the capacities of the
    r x r fine cells of a coarse cell sum to r^2 times its capacity)."""
    n, box, r = 10, 2.0, 4
    d = box / n
    x0, y0 = 20.0, 50.0
    cfg = W.base_config(nx=n, ny=n, x0=x0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1, num_levels=2,
                        ratios=[r], regrid_interval=3, patch_max=16, dt_max=30.0,
                        regions=[[x0 - 1, y0 - 1, x0 + box + 1, y0 + box + 1, 2, 2]])
    o = oracle.Oracle(cfg)
    o.add_topo(np.full((2, 2), -40.0), x0, y0, box, box)
    o.set_eta(0, *W.gaussian_grid(x0, y0, box, box, 41, 41, x0 + 0.8, y0 + 1.1, 1.0, 0.2, 0.3))
    o.init()
    o.step(4)
    h1, h2 = o.level_array(0, 1, "h"), o.level_array(0, 2, "h")
    k1 = np.array([_kappa(y0, d, J) for J in range(n)])[:, None]
    k2 = np.array([_kappa(y0, d / r, J) for J in range(n * r)])[:, None]
    m1 = np.sum(k1 * h1) * d * d
    m2 = np.sum(k2 * h2) * (d / r) * (d / r)
    assert abs(m1 - m2) <= 1e-12 * m2


def test_lonlat_workload_is_the_plane_workload_near_its_middle_latitude():
    """The latitude-longitude copy of a Cartesian workload (inputs mapped
    about the middle latitude) refines the same way and gives gauge records
    within the plane-limit difference (the domain spans ~2 degrees at 36 N,
    capacity varies by ~3% across it)."""
    wc = W.amr3(L=240e3, dx1=4000.0, steps=6)
    ws = W.lonlat(wc, lon0=142.0, lat0=35.0)
    cs = ws["cfg"]
    assert cs["spherical"] == 1 and cs["nx"] == wc["cfg"]["nx"]
    assert abs(cs["dy"] * R * D2R - wc["cfg"]["dx"]) < 1e-6
    phim = cs["y0"] + 0.5 * cs["ny"] * cs["dy"]
    assert abs(cs["dx"] * R * D2R * np.cos(phim * D2R) - wc["cfg"]["dx"]) < 1e-6
    a, b = W.load(oracle.Oracle(cs), ws), W.load(oracle.Oracle(wc["cfg"]), wc)
    a.step(6)
    b.step(6)
    assert a.stats()["cfl_violations"] == 0
    assert a.num_patches(0, 3) > 0
    assert abs(a.num_patches(0, 2) - b.num_patches(0, 2)) <= max(2, b.num_patches(0, 2) // 4)
    _, ea = a.read_gauges()
    _, eb = b.read_gauges()
    assert np.abs(ea - eb).max() <= 0.05 * np.abs(eb).max()


def test_time_step_from_capacity_scaled_speeds():
    """Still water over a flat bed at 30-40 N: every edge has the speed
    c = sqrt(g h).  After the first step dt comes from the sweeps' speeds:
    x edges of row J count c / kap_J, y edges c ced_e / kbar_e (reading of
    the capacity form's Courant numbers), so dt = 0.9 / max(c / (min kap dxp),
    c max(ced / kbar) / dyp) with dxp = dyp = R dphi."""
    n, d, depth = 20, 0.5, 3000.0
    y0 = 30.0
    cfg = W.base_config(nx=n, ny=n, x0=150.0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1)
    w = dict(cfg=cfg, topo=[(np.full((2, 2), -depth), 150.0, y0, n * d, n * d)], eta=[], uplift=[],
             gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    o.step(3)
    c = np.sqrt(9.81 * depth)
    kap = np.array([_kappa(y0, d, J) for J in range(-1, n + 1)])      # rows -1 .. n
    ced = np.cos((y0 + np.arange(0, n + 1) * d) * D2R)                # edges 0 .. n
    kbar = 0.5 * (kap[:-1] + kap[1:])                                  # edge e between rows e-1, e
    dp = R * d * D2R
    rate = max(c / (kap[1:-1].min() * dp), c * (ced / kbar).max() / dp)
    assert abs(o.stats()["dt"] - 0.9 / rate) <= 1e-12 * (0.9 / rate)
