"""Seeded synthetic inputs for the tsunami workloads.

This module only *generates inputs* (configuration dictionaries, bathymetry
grids, initial surfaces, seafloor uplift grids, gauge positions).  It holds
none of the method's arithmetic and imports nothing from the solver or the
oracle, so both can be driven from the same arrays.

The paper's benchmarks (2011 Tohoku, Seattle Fault; Sec. 5) need PMEL
deformation files, DEMs and tide records that are not available here.  These
generators stand in for them with the same structure: deep ocean, continental
slope, shelf, sloping beach and dry land, an instantaneous elliptical Gaussian
seafloor uplift, surface-elevation flagging and patch AMR with ratios 4-8.

Workloads (sizes in cells of level 1):
  hump200    200 x 200, dx = 10 m, flat 10 m, walls, Gaussian surface hump
             a = 0.5 m, sigma = 150 m at the centre, 100 steps, CFL 0.9.
  shelf(n)   n x n, dx = 500 m (4096 -> the 2048 km uniform run), shelf
             profile along x, 2 m uplift (sigma_x = 25 km, sigma_y = 50 km)
             600 km offshore, extrapolating boundaries.
  amr3(...)  3-level AMR over the shelf profile, ratios 4 and 4, flags
             |eta| > 0.01 m or depth < 200 m, regrid every 4 steps,
             patches up to 60 fine cells.
  amr4_bay   4-level AMR (ratios 4, 4, 8) down to 31.25 m around a synthetic
             semicircular bay on the beach, 10 gauges (deep, shelf, bay).
  ensemble   independent scenarios on one bathymetry, uplift centres and
             amplitudes drawn from numpy PCG64 with seed 1901.
  lonlat(w)  any of the above on a latitude-longitude grid (the coordinates
             of the paper's ocean runs): x and y in metres become longitude
             and latitude in degrees, cell sizes and input grids scaled to
             match at the domain's middle latitude.
"""
from __future__ import annotations

import numpy as np

BC_WALL, BC_EXTRAP = 0, 1


def base_config(**kw) -> dict:
    cfg = dict(nx=64, ny=64, x0=0.0, y0=0.0, dx=1.0, dy=1.0, num_levels=1, ratios=[], bc=[BC_WALL] * 4,
               g=9.81, drytol=1e-3, cfl_desired=0.9, cfl_max=1.0, dt_max=1e9, regrid_interval=0,
               flag_eta_tol=0.0, flag_depth_below=0.0, patch_max=64, level1_tile=0, regions=[],
               n_scenarios=1, transverse=0, cluster_eff=0.7, manning_n=0.0, spherical=0, earth_radius=0.0)
    cfg.update(kw)
    return cfg


def flat_topo(cfg: dict, depth: float):
    """A constant bed B = -depth covering the level-1 domain (2 x 2 grid)."""
    Lx, Ly = cfg["nx"] * cfg["dx"], cfg["ny"] * cfg["dy"]
    B = np.full((2, 2), -float(depth))
    return [(B, cfg["x0"], cfg["y0"], Lx, Ly)]


def gaussian_grid(x0, y0, Lx, Ly, n_x, n_y, xc, yc, amp, sx, sy):
    """Samples of amp * exp(-((x-xc)^2/(2 sx^2) + (y-yc)^2/(2 sy^2))) on an
    (n_y, n_x) node grid spanning [x0, x0+Lx] x [y0, y0+Ly]; returns the grid
    tuple (values, x0, y0, dx, dy)."""
    xs = x0 + np.arange(n_x) * (Lx / (n_x - 1))
    ys = y0 + np.arange(n_y) * (Ly / (n_y - 1))
    X, Y = np.meshgrid(xs, ys)
    v = amp * np.exp(-(((X - xc) / sx) ** 2 + ((Y - yc) / sy) ** 2) / 2.0)
    return (v, x0, y0, Lx / (n_x - 1), Ly / (n_y - 1))


def hump200() -> dict:
    """200 x 200, dx = 10 m, flat bottom depth 10 m, reflective walls, surface
    Gaussian hump 0.5 m, sigma 150 m at the centre, 100 steps at CFL 0.9."""
    cfg = base_config(nx=200, ny=200, dx=10.0, dy=10.0, bc=[BC_WALL] * 4, cfl_desired=0.9)
    eta = gaussian_grid(0.0, 0.0, 2000.0, 2000.0, 401, 401, 1000.0, 1000.0, 0.5, 150.0, 150.0)
    return dict(name="hump200", cfg=cfg, topo=flat_topo(cfg, 10.0), eta=[(0, *eta)], uplift=[], steps=100,
                gauges=np.array([[1000.0, 1000.0], [1500.0, 1000.0], [1000.0, 1700.0]]))


def shelf_profile_nodes(L_km: float, scale: float = 1.0, step_km: float = 1.0):
    """Bed elevation B(s) as a function of offshore distance s (km), with s
    measured from the x = L edge (the beach side).  Break points scale with
    ``scale``:  s in [0, 150]: +50 -> -200 m (shoreline at s = 30);
    [150, 450]: -200 m shelf; [450, 550]: -200 -> -4000 m slope; beyond: -4000 m.
    Returns node positions x (m) and values at spacing step_km*scale."""
    n = int(round(L_km / (step_km * scale))) + 1
    x_km = np.linspace(0.0, L_km, n)
    s = (L_km - x_km) / scale
    B = np.where(s <= 150.0, 50.0 - 250.0 * s / 150.0,
                 np.where(s <= 450.0, -200.0,
                          np.where(s <= 550.0, -200.0 - 3800.0 * (s - 450.0) / 100.0, -4000.0)))
    return x_km * 1000.0, B


def shelf_topo(Lx: float, Ly: float, scale: float = 1.0, step_km: float = 1.0):
    xs, B = shelf_profile_nodes(Lx / 1000.0, scale, step_km)
    grid = np.stack([B, B])
    return [(grid, 0.0, 0.0, xs[1] - xs[0], Ly)]


def shelf_uplift(Lx: float, Ly: float, scale: float = 1.0, amp: float = 2.0, s_km: float = 600.0,
                 yc: float | None = None, res: int = 4):
    """Elliptical Gaussian seafloor uplift: amp metres, sigma_x = 25 km
    (across the coast), sigma_y = 50 km (along it), centred s_km offshore.
    Sampled on a node grid covering +-4 sigma at ``res`` points per sigma_x."""
    sx, sy = 25e3 * scale, 50e3 * scale
    xc = Lx - s_km * 1e3 * scale
    yc = Ly / 2 if yc is None else yc
    x0, y0 = xc - 4 * sx, yc - 4 * sy
    nxg, nyg = 8 * res + 1, 8 * res * 2 + 1
    return gaussian_grid(x0, y0, 8 * sx, 8 * sy, nxg, nyg, xc, yc, amp, sx, sy)


def shelf(n: int = 4096, dx: float = 500.0, steps: int = 500) -> dict:
    """Uniform n x n grid over the shelf bathymetry with the 2 m uplift at
    t = 0 and extrapolating boundaries (the 4096^2, dx = 500 m run at n = 4096;
    smaller n crop the same physical layout at the same dx)."""
    L = n * dx
    scale = L / 2048e3
    cfg = base_config(nx=n, ny=n, dx=dx, dy=dx, bc=[BC_EXTRAP] * 4, cfl_desired=0.9)
    up = shelf_uplift(L, L, scale=scale)
    g = np.array([[L - 600e3 * scale, L / 2], [L - 300e3 * scale, L / 2], [L - 40e3 * scale, L / 2]])
    return dict(name=f"shelf{n}", cfg=cfg, topo=shelf_topo(L, L, scale=scale, step_km=max(1.0, dx / 1000.0)),
                eta=[], uplift=[(0, *up)], steps=steps, gauges=g)


def amr3(L: float = 2000e3, dx1: float = 2000.0, ratios=(4, 4), patch_max: int = 60,
         steps: int = 8, eta_tol: float = 0.01, depth_below: float = 200.0) -> dict:
    """3-level patch AMR over the shelf profile (ratios 4, 4), flags where
    |eta| > 0.01 m or depth < 200 m, regrid every 4 steps, patches up to 60
    fine cells per side (within the 16-64 range of the configuration; 60 is
    the column strip one 32-thread CTA of the FP32 update covers, so a patch
    row is one strip).  L = 2000 km, dx1 = 2 km is the full size; smaller L
    scales the bathymetry and uplift with the domain."""
    n = int(round(L / dx1))
    scale = L / 2000e3
    cfg = base_config(nx=n, ny=n, dx=dx1, dy=dx1, num_levels=len(ratios) + 1, ratios=list(ratios),
                      bc=[BC_EXTRAP] * 4, regrid_interval=4, flag_eta_tol=eta_tol,
                      flag_depth_below=depth_below, patch_max=patch_max)
    up = shelf_uplift(L, L, scale=scale)
    g = np.array([[L - 600e3 * scale, L / 2], [L - 300e3 * scale, L / 2], [L - 100e3 * scale, L / 2 + 10e3 * scale]])
    return dict(name="amr3", cfg=cfg, topo=shelf_topo(L, L, scale=scale, step_km=max(0.25, scale)),
                eta=[], uplift=[(0, *up)], steps=steps, gauges=g)


def bay_topo(L: float, scale: float, xs: float, yc: float, radius: float, box: float, res: float):
    """Fine topography grid over the bay box: the beach profile with a
    semicircular bay cut into it, B = min(B_beach, -10 (1 - (r / radius)^2))
    for r < radius around the shoreline point (xs, yc).  Node spacing res."""
    n = int(round(box / res)) + 1
    xg = xs - box / 2 + np.arange(n) * res
    yg = yc - box / 2 + np.arange(n) * res
    X, Y = np.meshgrid(xg, yg)
    s_km = (L - X) / 1000.0 / scale
    beach = np.where(s_km <= 150.0, 50.0 - 250.0 * s_km / 150.0, -200.0)
    r = np.hypot(X - xs, Y - yc)
    bay = np.where(r < radius, -10.0 * (1.0 - (r / radius) ** 2), np.inf)
    return (np.minimum(beach, bay), xg[0], yg[0], res, res)


def amr4_bay(L: float = 3000e3, dx1: float = 4000.0, ratios=(4, 4, 8), radius: float = 5000.0,
             box: float = 12000.0, patch_max: int = 60, eta_tol: float = 0.01, depth_below: float = 200.0,
             steps: int = 8) -> dict:
    """4-level AMR down to dx1 / 128 (31.25 m at full size) around a
    synthetic bay: the shelf profile scaled to the domain, a semicircular
    bay of the given radius cut into the beach at mid-y, the 2 m uplift of
    the uniform workload, flags |eta| > 0.01 m or depth < 200 m, the finest
    level forced over a box x box square around the bay and capped to three
    levels elsewhere, regrid every 4 steps, 10 gauges (4 deep water 700 km
    offshore, 3 on the shelf 300 km offshore, 3 in the bay; offsets scale
    with the domain)."""
    n = int(round(L / dx1))
    scale = L / 2048e3
    xs = L - 30e3 * scale                   # shoreline of the beach profile
    yc = L / 2
    nl = len(ratios) + 1
    half = box / 2
    bx1, by1, bx2, by2 = xs - half, yc - half, xs + half, yc + half
    big = 10 * L
    regions = [[bx1, by1, bx2, by2, nl, nl],                     # the bay box: finest level forced
               [-big, -big, bx1, big, 0, nl - 1], [bx2, -big, big, big, 0, nl - 1],   # elsewhere capped
               [bx1, -big, bx2, by1, 0, nl - 1], [bx1, by2, bx2, big, 0, nl - 1]]
    cfg = base_config(nx=n, ny=n, dx=dx1, dy=dx1, num_levels=nl, ratios=list(ratios), bc=[BC_EXTRAP] * 4,
                      regrid_interval=4, flag_eta_tol=eta_tol, flag_depth_below=depth_below,
                      patch_max=patch_max, regions=regions)
    up = shelf_uplift(L, L, scale=scale)
    finest = dx1
    for r in ratios:
        finest /= r
    topo = shelf_topo(L, L, scale=scale, step_km=max(0.25, scale)) + \
        [bay_topo(L, scale, xs, yc, radius, box, finest)]
    deep = [[L - 700e3 * scale, yc + d * scale] for d in (-300e3, -100e3, 100e3, 300e3)]
    shelfg = [[L - 300e3 * scale, yc + d * scale] for d in (-200e3, 0.0, 200e3)]
    bayg = [[xs - 0.4 * radius, yc], [xs + 0.4 * radius, yc - 0.4 * radius], [xs + 0.6 * radius, yc + 0.2 * radius]]
    return dict(name="amr4_bay", cfg=cfg, topo=topo, eta=[], uplift=[(0, *up)], steps=steps,
                gauges=np.array(deep + shelfg + bayg))


def ensemble(n_scen: int = 64, n: int = 1024, dx: float = 2000.0, ratio: int = 4, steps: int = 8,
             seed: int = 1901, patch_max: int = 60) -> dict:
    """Independent scenarios on one shelf bathymetry, 2 levels (ratio 4):
    uplift centres uniform over s in [550, 750] km x (mid +- 250 km) and
    amplitudes uniform in [0.5, 5] m, drawn from numpy PCG64(seed)."""
    L = n * dx
    scale = L / 2048e3
    rng = np.random.Generator(np.random.PCG64(seed))
    s_km = rng.uniform(550.0, 750.0, n_scen)
    yc = L / 2 + rng.uniform(-250e3, 250e3, n_scen) * scale
    amp = rng.uniform(0.5, 5.0, n_scen)
    cfg = base_config(nx=n, ny=n, dx=dx, dy=dx, num_levels=2, ratios=[ratio], bc=[BC_EXTRAP] * 4,
                      regrid_interval=4, flag_eta_tol=0.01, flag_depth_below=0.0, patch_max=patch_max,
                      n_scenarios=n_scen)
    ups = [(k, *shelf_uplift(L, L, scale=scale, amp=float(amp[k]), s_km=float(s_km[k]), yc=float(yc[k])))
           for k in range(n_scen)]
    g = np.array([[L - 650e3 * scale, L / 2], [L - 300e3 * scale, L / 2]])
    return dict(name=f"ensemble{n_scen}", cfg=cfg, topo=shelf_topo(L, L, scale=scale, step_km=max(1.0, dx / 1000)),
                eta=[], uplift=ups, steps=steps, gauges=g)


def dam_break_1d(n: int, hl: float, hr: float, L: float = 1000.0, ny: int = 4) -> dict:
    """Dam break on a flat bottom posed as a y-uniform 2D grid: depth hl for
    x < L/2 and hr beyond, at rest, walls far away (the run stops before any
    wave reaches them)."""
    dx = L / n
    cfg = base_config(nx=n, ny=ny, dx=dx, dy=dx, bc=[BC_EXTRAP, BC_EXTRAP, BC_WALL, BC_WALL], cfl_desired=0.9)
    topo = [(np.zeros((2, 2)), 0.0, 0.0, L, ny * dx)]
    # eta grid with a jump exactly between cells n/2-1 and n/2: nodes at cell centres
    xs = (np.arange(n) + 0.5) * dx
    row = np.where(xs < L / 2, hl, hr)
    eta = np.stack([row, row])
    return dict(name="dambreak", cfg=cfg, topo=topo, eta=[(0, eta, 0.5 * dx, 0.0, dx, ny * dx)], uplift=[],
                steps=0, gauges=np.zeros((0, 2)))


def lake_at_rest_shelf(n: int = 96, dx: float = 2000.0) -> dict:
    """Shelf bathymetry with beach and dry land, sea at rest (eta = 0)."""
    L = n * dx
    scale = L / 2048e3 * 4
    cfg = base_config(nx=n, ny=n, dx=dx, dy=dx, bc=[BC_EXTRAP] * 4)
    return dict(name="lake", cfg=cfg, topo=shelf_topo(L, L, scale=scale, step_km=max(0.25, scale)), eta=[],
                uplift=[], steps=0, gauges=np.zeros((0, 2)))


def cnn_init_params(seed: int = 0) -> np.ndarray:
    """Seeded starting weights of the refinement-flag predictor in the packed
    order of the C ABI (per layer 5->16, 16->16, 16->16 3x3 and 16->1 1x1:
    weights (out, in, k, k), then biases): He-normal weights from numpy
    PCG64(seed), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for ci, co, k in ((5, 16, 3), (16, 16, 3), (16, 16, 3), (16, 1, 1)):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (ci * k * k)), co * ci * k * k))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


def load(obj, w: dict):
    """Feed a workload's inputs to a solver object exposing add_topo,
    set_eta, set_velocity, add_uplift and init (the oracle or the GPU
    library binding)."""
    for (B, x0, y0, dx, dy) in w["topo"]:
        obj.add_topo(B, x0, y0, dx, dy)
    for (s, e, x0, y0, dx, dy) in w["eta"]:
        obj.set_eta(s, e, x0, y0, dx, dy)
    for (s, u, v, x0, y0, dx, dy) in w.get("uv", []):
        obj.set_velocity(s, u, v, x0, y0, dx, dy)
    for (s, d, x0, y0, dx, dy) in w["uplift"]:
        obj.add_uplift(s, d, x0, y0, dx, dy)
    if len(w.get("gauges", [])):
        obj.add_gauges(w["gauges"])
    obj.init()
    return obj


def lonlat(w: dict, lon0: float = 140.0, lat0: float = 30.0, radius: float = 6371.0e3) -> dict:
    """The workload ``w`` (Cartesian, metres) placed on a latitude-longitude
    grid: the point (x, y) goes to longitude lon0 + (x - x0) / (R cos(phi_m))
    and latitude lat0 + (y - y0) / R (in degrees; phi_m the domain's middle
    latitude), so the grid keeps its cell counts and, at phi_m, its cell sizes
    in metres.  Every input grid, region, uplift and gauge is mapped the same
    way; velocities stay in m/s.  Sets spherical = 1."""
    cfg = dict(w["cfg"])
    d2r = np.pi / 180.0
    ky = 1.0 / (radius * d2r)
    phim = lat0 + 0.5 * cfg["ny"] * cfg["dy"] * ky
    kx = 1.0 / (radius * d2r * np.cos(phim * d2r))
    xo, yo = cfg["x0"], cfg["y0"]

    def mx(x):
        return lon0 + (x - xo) * kx

    def my(y):
        return lat0 + (y - yo) * ky

    cfg.update(x0=lon0, y0=lat0, dx=cfg["dx"] * kx, dy=cfg["dy"] * ky, spherical=1, earth_radius=radius,
               regions=[[mx(r[0]), my(r[1]), mx(r[2]), my(r[3]), r[4], r[5]] for r in cfg.get("regions", [])])
    out = dict(w, cfg=cfg, name=w.get("name", "workload") + "_lonlat")
    out["topo"] = [(B, mx(x0), my(y0), dx * kx, dy * ky) for (B, x0, y0, dx, dy) in w["topo"]]
    out["eta"] = [(s, e, mx(x0), my(y0), dx * kx, dy * ky) for (s, e, x0, y0, dx, dy) in w["eta"]]
    out["uplift"] = [(s, d, mx(x0), my(y0), dx * kx, dy * ky) for (s, d, x0, y0, dx, dy) in w["uplift"]]
    out["uv"] = [(s, u, v, mx(x0), my(y0), dx * kx, dy * ky) for (s, u, v, x0, y0, dx, dy) in w.get("uv", [])]
    g = np.asarray(w.get("gauges", np.zeros((0, 2))), dtype=float).reshape(-1, 2)
    out["gauges"] = np.stack([mx(g[:, 0]), my(g[:, 1])], axis=1) if len(g) else g
    return out


def beach_runup(n: int = 48, ny: int = 12, cfl_retake: int = 1) -> dict:
    """A plane beach rising from 4 m depth at x = 0 to 4 m of dry land at
    x = L (shoreline mid-domain, dx = 5 m), a 1 m Gaussian surface hump
    (sigma 20 m) a quarter of the way in, uniform in y, walls: the wave runs
    up the dry half of the beach."""
    dx = 5.0
    L = n * dx
    cfg = base_config(nx=n, ny=ny, dx=dx, dy=dx, bc=[BC_WALL] * 4, cfl_desired=0.9, cfl_retake=cfl_retake)
    xs = np.linspace(0.0, L, 2 * n + 1)
    B = -4.0 + 8.0 * xs / L
    topo = [(np.vstack([B, B]), 0.0, 0.0, L / (2 * n), ny * dx)]
    eta = gaussian_grid(0.0, 0.0, L, ny * dx, 2 * n + 1, 5, 0.25 * L, 0.5 * ny * dx, 1.0, 20.0, 1e6)
    return dict(name="beach", cfg=cfg, topo=topo, eta=[(0, *eta)], uplift=[], steps=40, gauges=np.zeros((0, 2)))


def stepped_channel(seed: int, n: int = 40, ny: int = 2) -> dict:
    """A channel of n x ny unit cells between walls over a bed of random
    steps (every 5 cells, B uniform in [-3, 0.5] m), with a random surface
    (U(-0.5, 0.5) m) and velocity (U(-3, 3) m/s) per step section (numpy
    PCG64 seed): bed steps, dry cells, wetting and draining fronts and
    supersonic sections."""
    rng = np.random.default_rng(seed)
    cfg = base_config(nx=n, ny=ny, dx=1.0, dy=1.0, bc=[BC_WALL] * 4, cfl_desired=0.9)
    m = 4 * n + 1
    xs = np.linspace(0.0, n, m)
    seg = np.minimum(np.floor(xs / 5).astype(int), (m - 1) // 20)
    nseg = seg.max() + 1
    B = rng.uniform(-3, 0.5, nseg)[seg]
    eta = rng.uniform(-0.5, 0.5, nseg)[seg]
    u = rng.uniform(-3, 3, nseg)[seg]
    rows = ny + 1
    d = n / (m - 1)
    Bg, Eg, Ug = (np.tile(a, (rows, 1)) for a in (B, eta, u))
    return dict(name="channel", cfg=cfg, topo=[(Bg, 0.0, 0.0, d, 1.0)], eta=[(0, Eg, 0.0, 0.0, d, 1.0)],
                uv=[(0, Ug, np.zeros_like(Ug), 0.0, 0.0, d, 1.0)], uplift=[], steps=30, gauges=np.zeros((0, 2)))
