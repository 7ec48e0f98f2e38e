"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
closed forms (MC limiter table, the 1D dam-break solutions of Stoker and
Ritter), invariants the method must keep (lake at rest over bathymetry with
dry land, mass conservation between walls, mirror symmetry), exact
equalities the algorithm implies (one patch vs a tiled level; a fully
refined level vs a uniform fine grid; exact reproduction of linear data by
the interpolation) and hand-drawn clustering cases.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

G = 9.81


# --------------------------------------------------------------------------
# Riemann solver (Sec. 2.2; the paper only cites the solver, so its internals are a reading)

def _flux(h, hn, ht):
    """Physical flux of the x-split shallow water equations (Eq. swe)."""
    if h <= 0:
        return np.zeros(3)
    u = hn / h
    return np.array([hn, hn * u + 0.5 * G * h * h, hn * ht / h])


def test_riemann_equal_states_zero():
    rng = np.random.default_rng(0)
    for _ in range(200):
        h = rng.uniform(1e-2, 50)
        hn, ht, B = rng.normal(0, 5), rng.normal(0, 5), rng.uniform(-50, 0)
        Z, s, wl, wr = oracle.riemann(h, hn, ht, B, h, hn, ht, B)
        assert np.all(Z == 0.0)
        assert wl == 0 and wr == 0
    Z, s, wl, wr = oracle.riemann(0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 2.0)   # both dry
    assert np.all(Z == 0.0) and np.all(s == 0.0)


def test_riemann_lake_at_rest_exact():
    """Still water over any bed step (both wet) and at a dry shore: zero waves."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        BL, BR = -rng.uniform(0.01, 4000), -rng.uniform(0.01, 4000)
        Z, s, wl, wr = oracle.riemann(-BL, 0.0, 0.0, BL, -BR, 0.0, 0.0, BR)
        assert np.all(Z == 0.0)
    # wet cell next to dry land above the sea surface -> wall, still zero
    Z, s, wl, wr = oracle.riemann(3.0, 0.0, 0.0, -3.0, 0.0, 0.0, 0.0, 2.0)
    assert wr == 1 and np.all(Z == 0.0)
    Z, s, wl, wr = oracle.riemann(0.0, 0.0, 0.0, 5.0, 3.0, 0.0, 0.0, -3.0)
    assert wl == 1 and np.all(Z == 0.0)


def test_riemann_fwaves_sum_to_flux_jump_with_source():
    """f-wave decomposition: sum_p Z^p = f(Q_r) - f(Q_l) + g hbar (B_r - B_l)
    (the momentum source -g h B_x integrated across the edge)."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        hL, hR = rng.uniform(0.5, 100, 2)
        BL, BR = rng.uniform(-200, -110, 2)
        hnL, hnR, htL, htR = rng.normal(0, 20, 4)
        Z, s, wl, wr = oracle.riemann(hL, hnL, htL, BL, hR, hnR, htR, BR)
        df = _flux(hR, hnR, htR) - _flux(hL, hnL, htL)
        df[1] += G * 0.5 * (hL + hR) * (BR - BL)
        tot = Z.sum(axis=0)
        scale = np.abs(df).max() + 1.0
        assert np.allclose(tot, df, rtol=0, atol=1e-11 * scale), (tot, df)
        assert s[0] <= s[1] <= s[2]
        # Einfeldt-type bounds contain the characteristic speeds of both sides
        assert s[0] <= hnL / hL - math.sqrt(G * hL) + 1e-12
        assert s[2] >= hnR / hR + math.sqrt(G * hR) - 1e-12


def test_riemann_mirror_symmetry():
    """x -> -x: the problem (mirror R, mirror L) has speeds -s reversed and
    wave 1 <-> wave 3 with the normal-momentum component negated."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        hL, hR = rng.uniform(0.5, 60, 2)
        BL, BR = rng.uniform(-100, -70, 2)
        hnL, hnR, htL, htR = rng.normal(0, 10, 4)
        Z, s, _, _ = oracle.riemann(hL, hnL, htL, BL, hR, hnR, htR, BR)
        Zm, sm, _, _ = oracle.riemann(hR, -hnR, htR, BR, hL, -hnL, htL, BL)
        assert np.allclose(sm, -s[::-1], rtol=1e-14, atol=1e-14)
        flip = np.array([1.0, -1.0, 1.0])
        sc = np.abs(Z).max() + 1e-300
        assert np.allclose(Zm[0], Z[2] * flip, atol=1e-13 * sc)
        assert np.allclose(Zm[2], Z[0] * flip, atol=1e-13 * sc)
        assert np.allclose(Zm[1], Z[1] * flip, atol=1e-12 * sc)


def test_riemann_wall_no_mass_flux():
    """Against a wall the effective mass flux f(Q_l) + A-dQ vanishes."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        hL = rng.uniform(0.5, 5)
        uL = rng.uniform(-1, 1)
        Z, s, wl, wr = oracle.riemann(hL, hL * uL, 0.3 * hL, -hL, 0.0, 0.0, 0.0, 10.0)
        assert wr == 1
        amdq = sum(Z[p] * (1.0 if s[p] < 0 else (0.5 if s[p] == 0 else 0.0)) for p in range(3))
        assert abs(hL * uL + amdq[0]) < 1e-12


def test_riemann_dry_bed_front_speed():
    """Water next to a dry bed at the same level: the exact Riemann solution
    is a rarefaction whose front runs at u + 2c into a dry right side (u - 2c
    into a dry left side; Ritter's dam break), so the outermost wave speed is
    that front speed."""
    g = 9.81
    rng = np.random.default_rng(6)
    for _ in range(50):
        h, B = rng.uniform(0.1, 20.0), rng.uniform(-50.0, 0.0)
        u = rng.uniform(-1.0, 1.0) * np.sqrt(g * h)
        c = np.sqrt(g * h)
        _, s, wl, wr = oracle.riemann(h, h * u, 0.0, B, 0.0, 0.0, 0.0, B, g=g)
        assert wr == 0 and abs(s[2] - (u + 2.0 * c)) <= 1e-12 * (abs(u) + 2.0 * c)
        _, s, wl, wr = oracle.riemann(0.0, 0.0, 0.0, B, h, h * u, 0.0, B, g=g)
        assert wl == 0 and abs(s[0] - (u - 2.0 * c)) <= 1e-12 * (abs(u) + 2.0 * c)


def _shock_depth(h, u, g=9.81):
    """Depth behind the shock that stops a flow of depth h and speed u > 0 at
    a wall: (h* - h) sqrt(g (h* + h) / (2 h* h)) = u (Rankine-Hugoniot)."""
    lo, hi = h, 100.0 * h
    for _ in range(200):
        m = 0.5 * (lo + hi)
        if (m - h) * np.sqrt(g * (m + h) / (2.0 * m * h)) < u:
            lo = m
        else:
            hi = m
    return 0.5 * (lo + hi)


def test_riemann_flow_overtops_a_step_only_when_running_at_it():
    """Water of depth 1 m next to a dry step 2 m above its bed: at rest it
    cannot reach the step (a wall).  Running at the step at 3 m/s it piles
    up to the reflected-shock depth, 2.12 m, above the step, so water must
    cross (no wall); the solver's two-rarefaction estimate agrees here.
    Running away from the step it never crosses.  Mirrored for a step on the
    left."""
    h, step = 1.0, 2.0
    assert _shock_depth(h, 3.0) > step
    for u, wall in ((0.0, 1), (3.0, 0), (-3.0, 1)):
        _, _, wl, wr = oracle.riemann(h, h * u, 0.0, -5.0, 0.0, 0.0, 0.0, -5.0 + step)
        assert wr == wall, ("right", u)
        _, _, wl, wr = oracle.riemann(0.0, 0.0, 0.0, -5.0 + step, h, -h * u, 0.0, -5.0)
        assert wl == wall, ("left", u)


def test_riemann_single_shock_is_one_wave():
    """States joined by one 3-shock (Rankine-Hugoniot: s [h] = [hu],
    s [hu] = [hu^2 + g h^2 / 2]; right state at rest, depths 2 -> 1 and 3 -> 0.5,
    Lax-admissible) make one wave: for the shallow water equations the Roe
    average has the shock speed as an eigenvalue, so the Einfeldt bound
    s3 = max(u_r + c_r, u_hat + c_hat) is the shock speed and the whole flux
    jump goes into wave 3.  An unweighted velocity average (or any other
    average) leaves part of the jump in wave 1."""
    g = 9.81
    for hL, hR in ((2.0, 1.0), (3.0, 0.5)):
        # mass: s (hR - hL) = -hL uL; momentum: s (-hL uL) = g/2 (hR^2 - hL^2) - hL uL^2
        uL = math.sqrt(0.5 * g * (hL * hL - hR * hR) * (hL - hR) / (hL * hR))
        sh = hL * uL / (hL - hR)
        assert math.sqrt(g * hR) < sh < uL + math.sqrt(g * hL)    # Lax conditions (u_r = 0)
        Z, s, wl, wr = oracle.riemann(hL, hL * uL, 0.0, 0.0, hR, 0.0, 0.0, 0.0)
        assert s[2] == pytest.approx(sh, rel=1e-13)
        assert np.abs(Z[0]).max() <= 1e-12 * np.abs(Z[2]).max()
        assert np.abs(Z[2][:2] - np.array([-hL * uL, 0.5 * g * (hR * hR - hL * hL) - hL * uL * uL])).max() \
            <= 1e-12 * np.abs(Z[2]).max()


def test_square_pulse_makes_no_new_minimum():
    """A 0.1 m square pulse on 1 m of still water splits into two pulses.  The
    wave-limited scheme is TVD in each characteristic field of the linearised
    system, so the surface stays above the still level up to the nonlinear
    coupling (1e-3 m at this amplitude); a limiter fed the downwind neighbour
    undershoots by several millimetres."""
    n = 400
    cfg = W.base_config(nx=n, ny=4, dx=1.0, dy=1.0, bc=[W.BC_EXTRAP, W.BC_EXTRAP, W.BC_WALL, W.BC_WALL])
    xs = np.arange(n) + 0.5
    row = np.where((xs > 150) & (xs < 200), 1.1, 1.0)
    w = dict(cfg=cfg, topo=[(np.zeros((2, 2)), 0.0, 0.0, float(n), 4.0)],
             eta=[(0, np.stack([row, row]), 0.5, 0.0, 1.0, 4.0)], uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    o.step(60)
    h = o.level_array(0, 1, "h")
    assert h.min() > 1.0 - 1e-3
    assert h.max() < 1.1


def test_depth_flags_refine_the_shallow_band():
    """At rest, the only flags are depth < 200 m: after the first regrid every
    level-1 cell shallower than that is covered by level 2, and most of the
    covered area lies within the flag buffer of a shallow cell."""
    w = W.amr3(L=240e3, dx1=4000.0, steps=6)
    cfg = dict(w["cfg"], num_levels=2, ratios=[4], flag_eta_tol=0.0)
    w = dict(w, cfg=cfg, uplift=[])
    o = W.load(oracle.Oracle(cfg), w)
    B = o.level_array(0, 1, "B")
    shallow = -B < 200.0
    cov = np.zeros_like(shallow)
    for (i0, j0, nx, ny), _ in o.patches(0, 2):
        cov[j0 // 4:(j0 + ny) // 4, i0 // 4:(i0 + nx) // 4] = True
    assert shallow.any() and (~shallow).any()
    assert cov[shallow].all()
    b = cfg["regrid_interval"]
    near = np.zeros_like(shallow)
    for dj in range(-b, b + 1):
        for di in range(-b, b + 1):
            near |= np.roll(np.roll(shallow, dj, axis=0), di, axis=1)
    assert (cov & ~near).sum() <= 0.5 * cov.sum()


def test_mc_limiter_table():
    """MC limiter phi = max(0, min((1+t)/2, 2, 2t)) at tabulated points."""
    table = {-1.0: 0.0, 0.0: 0.0, 0.25: 0.5, 1 / 3: 2 / 3, 0.5: 0.75, 1.0: 1.0, 2.0: 1.5, 3.0: 2.0, 10.0: 2.0}
    for th, ph in table.items():
        assert oracle.mc_limiter(th) == pytest.approx(ph, rel=1e-15, abs=1e-15)


# --------------------------------------------------------------------------
# 1D dam break closed forms (posed as y-uniform 2D grids)

def _stoker_middle(hl, hr):
    """Middle state of the dam break: left rarefaction, right shock."""
    cl = math.sqrt(G * hl)

    def f(hm):
        u_raref = 2.0 * (cl - math.sqrt(G * hm))
        u_shock = (hm - hr) * math.sqrt(0.5 * G * (1.0 / hm + 1.0 / hr))
        return u_raref - u_shock
    a, b = hr, hl
    for _ in range(200):
        m = 0.5 * (a + b)
        if f(m) > 0:
            a = m
        else:
            b = m
    hm = 0.5 * (a + b)
    um = 2.0 * (cl - math.sqrt(G * hm))
    return hm, um


def dam_break_exact(x, t, x0, hl, hr):
    cl = math.sqrt(G * hl)
    xi = (x - x0) / t
    h = np.empty_like(x)
    if hr == 0.0:
        raref = (xi > -cl) & (xi < 2 * cl)
        h[:] = np.where(xi <= -cl, hl, 0.0)
        h[raref] = (2 * cl - xi[raref]) ** 2 / (9 * G)
        return h
    hm, um = _stoker_middle(hl, hr)
    cm = math.sqrt(G * hm)
    ss = hm * um / (hm - hr)
    h[:] = hl
    raref = (xi > -cl) & (xi < um - cm)
    h[raref] = (2 * cl - xi[raref]) ** 2 / (9 * G)
    h[(xi >= um - cm) & (xi < ss)] = hm
    h[xi >= ss] = hr
    return h


def _run_dam(n, hl, hr, T=40.0):
    w = W.dam_break_1d(n, hl, hr)
    o = W.load(oracle.Oracle(w["cfg"]), w)
    t = 0.0
    while t < T:
        t = o.step(1)[0]
    h = o.level_array(0, 1, "h")
    assert np.all(h == h[0:1, :]), "solution must stay uniform in y"
    dx = w["cfg"]["dx"]
    x = (np.arange(n) + 0.5) * dx
    ex = dam_break_exact(x, t, 500.0, hl, hr)
    return np.abs(h[0] - ex).sum() * dx / 1000.0


@pytest.mark.parametrize("hl,hr", [(2.0, 1.0), (1.0, 0.0)])
def test_dam_break_converges(hl, hr):
    errs = [_run_dam(n, hl, hr) for n in (100, 200, 400, 800)]
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert errs[-1] < 1e-2, errs
    assert np.mean(rates) >= 0.8, (errs, rates)


# --------------------------------------------------------------------------
# invariants of the 2D update

def test_hump_mass_and_mirror_symmetry():
    w = W.hump200()
    o = W.load(oracle.Oracle(w["cfg"]), w)
    m0 = o.stats()["mass"]
    o.step(100)
    st = o.stats()
    assert abs(st["mass"] - m0) <= 1e-13 * m0
    assert st["cfl_violations"] == 0
    h = o.level_array(0, 1, "h")
    assert np.abs(h - h[:, ::-1]).max() <= 1e-12 * np.abs(h).max()
    assert np.abs(h - h[::-1, :]).max() <= 1e-12 * np.abs(h).max()
    # transpose symmetry holds only to the splitting error (reported, loose bound)
    assert np.abs(h - h.T).max() < 1e-2


def test_mass_conservation_varying_bed():
    cfg = W.base_config(nx=60, ny=50, dx=50.0, dy=50.0, bc=[W.BC_WALL] * 4)
    xs = np.linspace(0, 3000, 61)
    B = -20.0 + 8.0 * np.sin(xs[None, :] / 400.0) * np.cos(np.linspace(0, 2500, 51)[:, None] / 300.0)
    eta = W.gaussian_grid(0, 0, 3000, 2500, 61, 51, 1200, 1400, 1.5, 300, 200)
    w = dict(cfg=cfg, topo=[(B, 0.0, 0.0, 50.0, 50.0)], eta=[(0, *eta)], uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    m0 = o.stats()["mass"]
    o.step(100)
    assert abs(o.stats()["mass"] - m0) <= 1e-13 * m0


def test_lake_at_rest_with_dry_land():
    """Still sea over the shelf profile with beach and dry land: nothing moves
    in 1000 steps."""
    w = W.lake_at_rest_shelf(n=96)
    o = W.load(oracle.Oracle(w["cfg"]), w)
    o.step(1000)
    for f in ("hu", "hv"):
        assert np.abs(o.level_array(0, 1, f)).max() == 0.0
    h = o.level_array(0, 1, "h")
    B = o.level_array(0, 1, "B")
    wet = h > 0
    assert np.abs((h + B)[wet]).max() == 0.0
    assert (~wet).sum() > 0 and wet.sum() > 0


def test_one_patch_equals_tiled_level():
    """Ghost fill by same-level copy: a tiled level 1 is bitwise the single patch
    after 100 steps, for tilings into uneven patches (37 and 64 cells with a
    ragged last row and column: 15 to 64 cells a side)."""
    w = W.hump200()
    a = W.load(oracle.Oracle(w["cfg"]), w)
    a.step(100)
    for tile, npatch in ((37, 36), (64, 16)):
        cfg = dict(w["cfg"], level1_tile=tile)
        b = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
        assert b.num_patches(0, 1) == npatch
        b.step(100)
        for f in ("h", "hu", "hv"):
            assert np.array_equal(a.level_array(0, 1, f), b.level_array(0, 1, f)), (tile, f)
        assert a.stats()["dt"] == b.stats()["dt"]
    # thin tiles next to the boundary: ghost cells past the domain edge of a
    # patch whose own side is not on it
    for bc in ([W.BC_WALL] * 4, [W.BC_EXTRAP] * 4):
        cfg = dict(w["cfg"], nx=9, ny=7, dx=200.0, dy=200.0, bc=bc)
        a = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
        cfg2 = dict(cfg, level1_tile=2)
        b = W.load(oracle.Oracle(cfg2), dict(w, cfg=cfg2))
        a.step(12)
        b.step(12)
        for f in ("h", "hu", "hv"):
            assert np.array_equal(a.level_array(0, 1, f), b.level_array(0, 1, f))


# --------------------------------------------------------------------------
# AMR

def test_interpolation_reproduces_linear_surface():
    """Minmod-limited linear interpolation is exact on a linear surface
    (pins the fine-cell offsets xi = ((I mod r) + 1/2)/r - 1/2)."""
    cfg = W.base_config(nx=24, ny=20, dx=100.0, dy=100.0, num_levels=2, ratios=[4], bc=[W.BC_EXTRAP] * 4,
                        regions=[[700.0, 500.0, 1700.0, 1500.0, 2, 2]], regrid_interval=0, patch_max=64)
    xs = np.linspace(0, 2400, 25)
    ys = np.linspace(0, 2000, 21)
    eta = 0.01 * xs[None, :] - 0.02 * ys[:, None] + 1.0
    w = dict(cfg=cfg, topo=[(np.full((2, 2), -50.0), 0.0, 0.0, 2400.0, 2000.0)],
             eta=[(0, eta, 0.0, 0.0, 100.0, 100.0)], uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    pats = o.patches(0, 2)
    assert len(pats) >= 1
    dxf = 25.0
    for (i0, j0, nx, ny), a in pats:
        x = (i0 + np.arange(nx) + 0.5) * dxf
        y = (j0 + np.arange(ny) + 0.5) * dxf
        exact = 0.01 * x[None, :] - 0.02 * y[:, None] + 1.0
        assert np.abs(a["h"] + a["B"] - exact).max() < 1e-12


def test_amr_lake_at_rest():
    """Still sea under 3-level AMR with regridding every 2 steps: exactly at rest
    on every level after 63 coarse steps (1008 steps of the finest level)."""
    w = W.amr3(L=120e3, dx1=4000.0, steps=8, eta_tol=0.01, depth_below=200.0)
    cfg = dict(w["cfg"], regrid_interval=2)
    w = dict(w, cfg=cfg, uplift=[])
    o = W.load(oracle.Oracle(cfg), w)
    assert o.num_patches(0, 2) > 0 and o.num_patches(0, 3) > 0
    o.step(63)
    assert o.num_patches(0, 2) > 0 and o.num_patches(0, 3) > 0
    for lev in (1, 2, 3):
        for box, a in o.patches(0, lev):
            assert np.abs(a["hu"]).max() == 0.0 and np.abs(a["hv"]).max() == 0.0
            wet = a["h"] > 0
            assert np.abs((a["h"] + a["B"])[wet]).max() == 0.0


def _fixed_dt_cfg(cfg, dt):
    c = dict(cfg)
    c["dt_max"] = dt
    c["cfl_desired"] = 0.9
    return c


def test_full_coverage_level2_equals_uniform_fine():
    """Level 2 covering the whole domain (forced region) evolves exactly like
    a uniform grid at the fine resolution with the same time steps."""
    nx, dx, r = 16, 400.0, 4
    L = nx * dx
    base = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_WALL] * 4)
    topo = [(np.array([[-30.0, -10.0], [-30.0, -10.0]]), 0.0, 0.0, L, L)]
    up = W.gaussian_grid(0.0, 0.0, L, L, 65, 65, 3000.0, 3400.0, 0.8, 700.0, 500.0)
    dt = 2.0
    amr_cfg = _fixed_dt_cfg(dict(base, num_levels=2, ratios=[r], regrid_interval=2, patch_max=24,
                                 regions=[[-1.0, -1.0, L + 1, L + 1, 2, 2]]), dt)
    fine_cfg = _fixed_dt_cfg(W.base_config(nx=nx * r, ny=nx * r, dx=dx / r, dy=dx / r, bc=[W.BC_WALL] * 4,
                                           level1_tile=29), dt / r)
    a = oracle.Oracle(amr_cfg)
    b = oracle.Oracle(fine_cfg)
    for o in (a, b):
        o.add_topo(*topo[0])
        o.init()
        o.add_uplift(0, *up)
    for _ in range(3):
        a.step(1)
        b.step(r)
    assert a.stats()["cfl_violations"] == 0
    for f in ("h", "hu", "hv"):
        assert np.array_equal(a.level_array(0, 2, f), b.level_array(0, 1, f))


def test_averaging_conserves_mass_flat_bed():
    """Full coverage over a flat bed with no dry cells: the averaged level-1
    mass equals the level-2 mass."""
    nx, dx, r = 12, 300.0, 4
    L = nx * dx
    cfg = _fixed_dt_cfg(W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_WALL] * 4, num_levels=2,
                                      ratios=[r], regrid_interval=3, patch_max=16,
                                      regions=[[-1.0, -1.0, L + 1, L + 1, 2, 2]]), 1.5)
    o = oracle.Oracle(cfg)
    o.add_topo(np.full((2, 2), -20.0), 0.0, 0.0, L, L)
    o.set_eta(0, *W.gaussian_grid(0, 0, L, L, 49, 49, 1500, 2000, 1.0, 400, 300))
    o.init()
    o.step(4)
    m1 = np.nansum(o.level_array(0, 1, "h")) * dx * dx
    m2 = np.nansum(o.level_array(0, 2, "h")) * (dx / r) ** 2
    assert abs(m1 - m2) <= 1e-12 * m2


def test_partial_refinement_closer_to_fine_than_coarse():
    """A refined patch around a wave is closer to the uniform fine solution
    than the coarse grid is (space-time interpolation at its boundary)."""
    nx, dx, r = 24, 400.0, 4
    L = nx * dx
    topo = (np.full((2, 2), -40.0), 0.0, 0.0, L, L)
    up = W.gaussian_grid(0.0, 0.0, L, L, 97, 97, 4800.0, 4800.0, 1.0, 900.0, 900.0)
    reg = [[2400.0, 2400.0, 7200.0, 7200.0, 2, 2]]
    dt = 3.0
    amr = _fixed_dt_cfg(W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, num_levels=2, ratios=[r], patch_max=64,
                                      regrid_interval=0, regions=reg), dt)
    crs = _fixed_dt_cfg(W.base_config(nx=nx, ny=nx, dx=dx, dy=dx), dt)
    fin = _fixed_dt_cfg(W.base_config(nx=nx * r, ny=nx * r, dx=dx / r, dy=dx / r), dt / r)
    runs = []
    for cfg, k in ((amr, 1), (crs, 1), (fin, r)):
        o = oracle.Oracle(cfg)
        o.add_topo(*topo)
        o.init()
        o.add_uplift(0, *up)
        for _ in range(6):
            o.step(k)
        runs.append(o)
    a, c, f = runs
    xs = np.arange(3000.0, 6600.0, 100.0) + 12.5
    fa = a.read_field(0, 0, "eta", len(xs), len(xs), xs[0], xs[0], 100.0, 100.0)
    fc = c.read_field(0, 0, "eta", len(xs), len(xs), xs[0], xs[0], 100.0, 100.0)
    ff = f.read_field(0, 0, "eta", len(xs), len(xs), xs[0], xs[0], 100.0, 100.0)
    assert np.abs(fa - ff).max() < 0.5 * np.abs(fc - ff).max()


def test_time_interpolation_of_ghosts_on_a_sloped_surface():
    """Coarse-to-fine ghost values are linear in time within a coarse step
    (Sec. 3.1 step 2: between the coarse states before and after its step).  Still water under a uniform surface
    slope s accelerates uniformly: hu = -g h s t, while eta changes only at
    O(s^2).  So linear space-time interpolation of the coarse state is exact up
    to those terms, and a refined band across the domain must match the
    uniform fine grid after 4 coarse steps to 5e-5 of the momentum (measured
    1.3e-5).  A time fraction off by part of a coarse step misses by 1e-4 to
    1e-1: the fraction reversed in the depth only (2.3e-4), or the ghosts
    taken from the old or the new coarse state alone (0.08-0.1)."""
    nx, ny, dx, r, dt, s, depth = 48, 16, 400.0, 4, 16.0, 1e-4, 40.0
    L, Ly = nx * dx, ny * dx
    topo = (np.full((2, 2), -depth), 0.0, 0.0, L, Ly)
    xs = np.linspace(0.0, L, 4 * nx + 1)
    eta = np.tile(s * (xs - L / 2), (4 * ny + 1, 1))
    band = [[6400.0, 0.0, 12800.0, Ly, 2, 2]]           # level 2 over x in [6.4, 12.8] km, all y
    bc = [W.BC_EXTRAP] * 4
    amr = _fixed_dt_cfg(W.base_config(nx=nx, ny=ny, dx=dx, dy=dx, num_levels=2, ratios=[r], patch_max=64,
                                      regrid_interval=0, regions=band, bc=bc), dt)
    fin = _fixed_dt_cfg(W.base_config(nx=nx * r, ny=ny * r, dx=dx / r, dy=dx / r, bc=bc), dt / r)
    runs = []
    for cfg, k in ((amr, 1), (fin, r)):
        o = oracle.Oracle(cfg)
        o.add_topo(*topo)
        o.set_eta(0, eta, 0.0, 0.0, L / (4 * nx), Ly / (4 * ny))
        o.init()
        for _ in range(4):
            o.step(k)
        runs.append(o)
    a, f = runs
    assert a.num_patches(0, 2) > 0
    fx = dx / r
    x = np.arange(6400.0, 12800.0, fx) + fx / 2           # the whole band ...
    y = np.arange(0.25 * Ly, 0.75 * Ly, fx) + fx / 2      # ... away from the y boundaries
    for fld in ("hu", "eta"):
        fa = a.read_field(0, 0, fld, len(x), len(y), x[0], y[0], fx, fx)
        ff = f.read_field(0, 0, fld, len(x), len(y), x[0], y[0], fx, fx)
        assert np.abs(fa - ff).max() <= 5e-5 * np.abs(ff).max(), fld
    # the band does accelerate: hu = -g h s t to within the O(s^2) terms
    hu = a.read_field(0, 0, "hu", len(x), len(y), x[0], y[0], fx, fx)
    expect = -9.81 * depth * s * (4 * dt)
    assert np.abs(hu - expect).max() <= 0.02 * abs(expect)


# --------------------------------------------------------------------------
# clustering (Sec. 3.2, Berger & Rigoutsos)

def _check_boxes(flags, boxes, pm=None):
    ny, nx = flags.shape
    cover = np.zeros_like(flags, dtype=int)
    for i0, j0, w, h in boxes:
        assert w > 0 and h > 0 and i0 >= 0 and j0 >= 0 and i0 + w <= nx and j0 + h <= ny
        if pm is not None:
            assert w <= pm and h <= pm
        cover[j0:j0 + h, i0:i0 + w] += 1
    assert cover.max() <= 1, "boxes overlap"
    assert np.all(cover[flags.astype(bool)] == 1), "a flag is not covered"


def test_cluster_single_rectangle():
    f = np.zeros((20, 30), np.uint8)
    f[3:9, 5:17] = 1
    b = oracle.cluster(f)
    assert b.tolist() == [[5, 3, 12, 6]]


def test_cluster_hole_cut():
    f = np.zeros((10, 20), np.uint8)
    f[2:6, 1:5] = 1
    f[2:6, 12:16] = 1
    b = oracle.cluster(f)
    assert sorted(b.tolist()) == [[1, 2, 4, 4], [12, 2, 4, 4]]


def test_cluster_L_shape_and_random_invariants():
    f = np.zeros((16, 16), np.uint8)
    f[0:12, 0:3] = 1
    f[9:12, 0:14] = 1
    b = oracle.cluster(f)
    _check_boxes(f, b)
    assert len(b) >= 2
    for i0, j0, w, h in b:
        assert f[j0:j0 + h, i0:i0 + w].mean() >= 0.7
    rng = np.random.default_rng(7)
    for _ in range(60):
        f = (rng.random((23, 31)) < rng.uniform(0.02, 0.4)).astype(np.uint8)
        b = oracle.cluster(f, ratio=4, patch_max=24)
        _check_boxes(f, b, pm=6)


def test_cluster_respects_nesting():
    f = np.zeros((12, 12), np.uint8)
    f[1, 1] = 1
    f[10, 10] = 1
    f[1, 10] = 1
    nest = np.ones_like(f)
    nest[5:8, 5:8] = 0
    b = oracle.cluster(f, nest, eff=0.0)
    _check_boxes(f, b)
    for i0, j0, w, h in b:
        assert nest[j0:j0 + h, i0:i0 + w].all()


def test_cluster_cut_rules_worked_by_hand():
    """The clustering reading (Berger-Rigoutsos, Sec. 3.2) applied by hand to
    masks where each rule decides the outcome; the expected boxes are derived
    in the comments, not taken from the code.

    (a) Acceptance is flags >= eff * area: a row of 8 with 4 flags at
        eff = 0.5 is one box (a strict test would cut it in two).
    (b) Of two holes, the cut goes through the one nearest the box centre: a
        row of 11 with holes at 1 and 4 (centre 5), eff = 0.85.  Cut at 4:
        left 0..3 holds 3 of 4 (< 0.85) and is cut at its hole 1 into [0] and
        [2, 3]; right 5..10 is full.  (Cutting at 1 first would leave 2..10,
        8 of 9 >= 0.85, as one box.)
    (c) The lower / left part is clustered first: two rectangles come out
        left, then right.
    (d) Without holes, the cut goes at the strongest sign change of the
        signature's Laplacian, ties to the one nearer the centre.  Column
        heights 1 1 2 1 2 1 (2 rows, 8 of 12, eff 0.7): Laplacian 1 -2 2 -2,
        sign changes of strength 3, 4, 4 between columns 1|2, 2|3, 3|4; the
        tie goes to 2|3 (at the centre).  Each half (3 wide, 4 of 6) has no
        hole and no inflection and is bisected at 0|1 and 3|4, leaving [0],
        [1, 2] x 2 rows, [3], [4, 5] x 2 rows (3 of 4 each, accepted).  (The
        weakest change, 1|2, would give [0, 1] and [2..5] x 2 rows.)"""
    f = np.array([[1, 1, 0, 0, 0, 0, 1, 1]], np.uint8)
    assert oracle.cluster(f, eff=0.5).tolist() == [[0, 0, 8, 1]]
    f = np.array([[1, 0, 1, 1, 0, 1, 1, 1, 1, 1, 1]], np.uint8)
    assert oracle.cluster(f, eff=0.85).tolist() == [[0, 0, 1, 1], [2, 0, 2, 1], [5, 0, 6, 1]]
    f = np.zeros((10, 20), np.uint8)
    f[2:6, 12:16] = 1
    f[2:6, 1:5] = 1
    assert oracle.cluster(f).tolist() == [[1, 2, 4, 4], [12, 2, 4, 4]]
    f = np.array([[1, 1, 1, 1, 1, 1], [0, 0, 1, 0, 1, 0], [0, 0, 0, 0, 0, 0]], np.uint8)
    assert oracle.cluster(f, eff=0.7).tolist() == [[0, 0, 1, 1], [1, 0, 2, 2], [3, 0, 1, 1], [4, 0, 2, 2]]


def test_cluster_splits_large_boxes_into_near_equal_pieces_row_by_row():
    """A box wider or taller than patch_max (in fine cells) is cut into the
    fewest pieces that fit, ceil(w / pm) x ceil(h / pm) with pm = patch_max /
    ratio coarse cells; the widths (and heights) differ by at most one; the
    pieces tile the box and come out row by row."""
    for (w, h, ratio, patch_max) in ((10, 7, 2, 8), (13, 5, 4, 16), (9, 9, 1, 3), (17, 4, 2, 10)):
        f = np.zeros((h + 3, w + 4), np.uint8)
        f[1:1 + h, 2:2 + w] = 1
        b = oracle.cluster(f, ratio=ratio, patch_max=patch_max).tolist()
        pm = patch_max // ratio
        npx, npy = -(-w // pm), -(-h // pm)
        assert len(b) == npx * npy
        cover = np.zeros_like(f, int)
        for i0, j0, bw, bh in b:
            assert bw <= pm and bh <= pm
            cover[j0:j0 + bh, i0:i0 + bw] += 1
        assert np.array_equal(cover, f.astype(int))
        widths = [bw for _, _, bw, _ in b[:npx]]
        heights = [bh for _, _, _, bh in b[::npx]]
        assert max(widths) - min(widths) <= 1 and max(heights) - min(heights) <= 1
        assert [(j0, i0) for i0, j0, _, _ in b] == sorted((j0, i0) for i0, j0, _, _ in b)   # row by row


def test_interpolation_makes_no_new_extrema():
    """A limited linear reconstruction keeps every fine value inside the range
    of its coarse cell and the neighbours (no new extrema).  Coarse surface
    with a kink: slope 0.02 per cell, then 0.08; the cell at the kink has
    one-sided differences in a ratio of 4, where a slope larger than the
    smaller difference would push its outer fine cells past a neighbour."""
    nx, ny, dx = 40, 8, 100.0
    i = np.arange(nx)
    eta_c = np.where(i < 20, 0.02 * i, 0.4 + 0.08 * (i - 20))
    cfg = W.base_config(nx=nx, ny=ny, dx=dx, dy=dx, bc=[W.BC_EXTRAP] * 4, num_levels=2, ratios=[4],
                        regrid_interval=4, regions=[[1200.0, 0.0, 2800.0, ny * dx, 2, 2]])
    w = dict(cfg=cfg, topo=[(np.full((2, 2), -100.0), 0.0, 0.0, nx * dx, ny * dx)],
             eta=[(0, np.stack([eta_c, eta_c]), 0.5 * dx, 0.0, dx, ny * dx)], uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    e1, e2 = o.level_array(0, 1, "eta"), o.level_array(0, 2, "eta")
    assert np.abs(e1[3] - eta_c).max() < 1e-12
    checked = 0
    for J, I in zip(*np.nonzero(~np.isnan(e2))):
        Ic, Jc = I // 4, J // 4
        nb = e1[max(Jc - 1, 0):Jc + 2, max(Ic - 1, 0):Ic + 2]
        assert nb.min() - 1e-12 <= e2[J, I] <= nb.max() + 1e-12, (I, J, e2[J, I], nb.min(), nb.max())
        checked += 1
    assert checked > 0 and not np.isnan(e2[:, 80:84]).all()    # the kink cell is refined
