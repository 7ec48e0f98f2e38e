"""Pins of the oracle's AMR bookkeeping (Sec. 3.1-3.2, Sec. 5.1.2), each
against a definition or a closed form rather than against the oracle's own
arithmetic:

* updating (Sec. 3.1 step 4): after a coarse step, a coarse cell under a
  fine patch holds the mean of the fine momenta and, where a fine cell is
  wet, the mean surface of the wet fine cells (h = max(0, eta - B));
* the time step (nu over the largest Courant rate of any level; the first
  step takes its rates from the cells): for uniform flow over a flat bed it is
  nu * min(dx / (|u| + c), dy / (|v| + c)) exactly, and the next step (from
  the edges' wave speeds) gives the same; over levels it follows the fastest
  (a trench only level 2 resolves sets it);
* the flag criterion (Sec. 3.2): every cell with |eta| above the tolerance,
  crest or trough, lies under a finer patch after a regrid;
* the flag buffer (Sec. 3.2; b cells, b the regrid interval): a single
  flagged cell refines exactly its (2b + 1)^2 Chebyshev neighbourhood;
* proper nesting (Sec. 3.1: fine ghost cells come from the next coarser
  level): a level-3 patch stays 2 level-2 cells inside level 2, at every step
  of a run with regrids;
* gauges (Sec. 5.1.2): on a frozen linear surface a gauge reads the surface
  exactly; on a quadratic one its error stays within the finest level's
  bilinear interpolation bound, 16 times below the coarse level's;
* seafloor uplift (Sec. 5.1.1): given before or after init, it raises B by
  dB on every level and keeps h and the mass, so eta rises by dB where wet;
* the zeta field (Sec. 5.1.2, Eq. zeta): for a still sea at +0.5 m over a
  beach, 0.5 offshore, 0.5 - B on flooded land and 0 above, the closed form
  that zeta = eta or zeta = h everywhere (both planted, both caught) miss.

A throwaway mutation run planted one mistake at a time in oracle/amr.c. Each
of the ten below passed every earlier pin, and each fails one here: momentum
averaging skipped; eta averaged over dry cells too; the cell speed without the
velocity, or with u and v swapped; flags on eta > tol instead of |eta| > tol;
a buffer of b - 1 cells; a nesting margin of 1 cell; gauges from the nearest
cell, from the coarsest level, or without the half-cell offset.  Three uplift
mistakes (the surface left in place at init, fine levels' B without the
uplift, a late uplift that also lowers h) were caught before only in passing,
by tests about other things; the uplift pin catches each directly.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W


# --------------------------------------------------------------------------
# updating (fine-to-coarse averaging)

def test_coarse_cells_under_fine_patches_hold_the_fine_averages():
    """A 2-level shelf with uplift, beach and dry land; level 2 forced over a
    band that spans deep water, the shoreline and dry land, no regrids (so
    no patch is rebuilt between the averaging and the check).  The sea stands
    at +0.5 m (still water at any constant level is at rest), so the wet fine
    cells of a coarse cell across the shoreline carry a surface that is not 0
    and the mean over wet cells differs from a mean over all of them."""
    w = W.shelf(n=96, dx=4000.0, steps=12)             # the shoreline falls inside a coarse cell
    L = 96 * 4000.0
    r = 4
    band = [[0.45 * L, 0.2 * L, L, 0.8 * L, 2, 2]]
    cfg = dict(w["cfg"], num_levels=2, ratios=[r], regrid_interval=0, regions=band, patch_max=32)
    sea = [(0, np.full((2, 2), 0.5), 0.0, 0.0, L, L)]
    o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg, eta=sea))
    o.step(12)
    drytol = cfg["drytol"]
    coarse = {f: o.level_array(0, 1, f) for f in ("h", "hu", "hv", "B")}
    n_checked = n_partial = 0
    mom_scale = max(np.nanmax(np.abs(coarse["hu"])), np.nanmax(np.abs(coarse["hv"])))
    assert mom_scale > 0.0
    for box, a in o.patches(0, 2):
        i0, j0, nx, ny = box
        for Jc in range(j0 // r, (j0 + ny) // r):
            for Ic in range(i0 // r, (i0 + nx) // r):
                sl = (slice(Jc * r - j0, Jc * r - j0 + r), slice(Ic * r - i0, Ic * r - i0 + r))
                hf, Bf = a["h"][sl], a["B"][sl]
                wet = hf >= drytol
                hc, Bc = coarse["h"][Jc, Ic], coarse["B"][Jc, Ic]
                if wet.any():
                    eta_bar = (hf + Bf)[wet].mean()
                    assert abs(hc - max(0.0, eta_bar - Bc)) <= 1e-12 * max(1.0, abs(Bc)), (Ic, Jc)
                    n_partial += int(not wet.all())
                else:
                    assert hc == 0.0
                if hc >= drytol:
                    for f in ("hu", "hv"):
                        assert abs(coarse[f][Jc, Ic] - a[f][sl].mean()) <= 1e-12 * mom_scale, (f, Ic, Jc)
                else:
                    assert coarse["hu"][Jc, Ic] == 0.0 and coarse["hv"][Jc, Ic] == 0.0
                n_checked += 1
    assert n_checked > 100
    assert n_partial > 0        # coarse cells across the shoreline: wet and dry fine cells


# --------------------------------------------------------------------------
# the first time step

def test_first_time_step_of_uniform_flow_on_2_to_1_cells():
    u0, v0, depth, dx, dy, nu = 2.0, -5.0, 10.0, 100.0, 50.0, 0.9
    cfg = W.base_config(nx=24, ny=48, dx=dx, dy=dy, bc=[W.BC_EXTRAP] * 4, cfl_desired=nu)
    Lx, Ly = 24 * dx, 48 * dy
    U = np.full((3, 3), u0)
    V = np.full((3, 3), v0)
    w = dict(cfg=cfg, topo=W.flat_topo(cfg, depth), eta=[], uplift=[], gauges=np.zeros((0, 2)),
             uv=[(0, U, V, 0.0, 0.0, Lx / 2, Ly / 2)])
    o = W.load(oracle.Oracle(cfg), w)
    c = np.sqrt(9.81 * depth)
    expect = nu * min(dx / (abs(u0) + c), dy / (abs(v0) + c))
    t1 = o.step(1)[0]
    assert abs(t1 - expect) <= 1e-14 * expect
    t2 = o.step(1)[0]
    assert abs((t2 - t1) - expect) <= 1e-12 * expect
    # the flow stays uniform, so nothing else changed
    assert np.allclose(o.level_array(0, 1, "hu"), depth * u0, rtol=1e-13, atol=0.0)


def test_time_step_follows_the_fastest_level():
    """Reading c7 over levels: dt = nu / max_l(rate_l / R_l), R_l the steps a
    level takes per coarse step.  A 100 m trench narrower than a coarse cell
    and between coarse centres is seen only by level 2 (each level samples
    the bed at its own centres), so still water gives the first step
    nu dx1 / sqrt(g 100) from level 2, not nu dx1 / sqrt(g 10) from level 1;
    no step then exceeds Courant 1 on any level."""
    nx, dx, r, nu, g = 16, 1000.0, 4, 0.9, 9.81
    L = nx * dx
    xs = np.arange(0.0, L + 1.0, dx / 16)
    B = np.where((xs >= 1000.0) & (xs <= 1250.0), -100.0, -10.0)
    bed = np.tile(B, (17, 1))
    cfg = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_WALL] * 4, num_levels=2, ratios=[r], cfl_desired=nu,
                        regrid_interval=0, regions=[[0.0, 0.0, 3000.0, L, 2, 2]])
    w = dict(cfg=cfg, topo=[(bed, 0.0, 0.0, dx / 16, L / 16)], eta=[], uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    assert np.nanmax(o.level_array(0, 1, "h")) == 10.0                  # level 1 never sees the trench
    assert max(a["h"].max() for _, a in o.patches(0, 2)) == 100.0
    t1 = o.step(1)[0]
    expect = nu * dx / np.sqrt(g * 100.0)
    assert abs(t1 - expect) <= 1e-13 * expect
    o.step(20)
    assert o.stats()["cfl_violations"] == 0


# --------------------------------------------------------------------------
# flagging, buffer, nesting

def _deep_basin(nx, dx, levels, r, b, eta_grid=None, regions=None, eta_tol=0.0):
    cfg = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_EXTRAP] * 4, num_levels=levels,
                        ratios=[r] * (levels - 1), regrid_interval=b, flag_eta_tol=eta_tol,
                        regions=regions or [], patch_max=64)
    eta = [] if eta_grid is None else [(0, *eta_grid)]
    return cfg, dict(cfg=cfg, topo=W.flat_topo(cfg, 4000.0), eta=eta, uplift=[], gauges=np.zeros((0, 2)))


def test_crests_and_troughs_are_both_refined():
    nx, dx = 64, 1000.0
    L = nx * dx
    crest = W.gaussian_grid(0, 0, L, L, 257, 257, 0.3 * L, 0.5 * L, 0.5, 3000.0, 3000.0)
    trough = W.gaussian_grid(0, 0, L, L, 257, 257, 0.7 * L, 0.5 * L, -0.5, 3000.0, 3000.0)
    eta = (crest[0] + trough[0], *crest[1:])
    cfg, w = _deep_basin(nx, dx, 2, 4, 2, eta_grid=eta, eta_tol=0.01)
    o = W.load(oracle.Oracle(cfg), w)
    e = o.level_array(0, 1, "eta")
    covered = np.zeros((nx, nx), bool)
    for (i0, j0, bw, bh), _ in o.patches(0, 2):
        covered[j0 // 4:(j0 + bh) // 4, i0 // 4:(i0 + bw) // 4] = True
    hi = np.abs(e) > 0.01
    assert (e > 0.01).any() and (e < -0.01).any()
    assert covered[hi].all()


@pytest.mark.parametrize("b", [2, 3, 4])
def test_one_flagged_cell_refines_its_buffer_exactly(b):
    nx, dx, r = 40, 1000.0, 2
    ic, jc = 17, 22                                   # the flagged cell
    x, y = (ic + 0.5) * dx, (jc + 0.5) * dx
    reg = [[x - 0.1 * dx, y - 0.1 * dx, x + 0.1 * dx, y + 0.1 * dx, 2, 2]]   # holds only that centre
    cfg, w = _deep_basin(nx, dx, 2, r, b, regions=reg)
    o = W.load(oracle.Oracle(cfg), w)
    covered = np.zeros((nx, nx), bool)
    for (i0, j0, bw, bh), _ in o.patches(0, 2):
        assert i0 % r == 0 and j0 % r == 0 and bw % r == 0 and bh % r == 0
        covered[j0 // r:(j0 + bh) // r, i0 // r:(i0 + bw) // r] = True
    expect = np.zeros((nx, nx), bool)
    expect[jc - b:jc + b + 1, ic - b:ic + b + 1] = True
    assert np.array_equal(covered, expect)


def _nesting_violations(o, nxl2, nyl2, r2):
    """Level-2 cells within 2 cells (Chebyshev) of a level-3 patch's footprint
    that no level-2 patch covers (inside the domain)."""
    cov2 = np.zeros((nyl2, nxl2), bool)
    for (i0, j0, bw, bh), _ in o.patches(0, 2):
        cov2[j0:j0 + bh, i0:i0 + bw] = True
    bad = 0
    for (i0, j0, bw, bh), _ in o.patches(0, 3):
        I0, J0, I1, J1 = i0 // r2, j0 // r2, (i0 + bw) // r2, (j0 + bh) // r2
        win = cov2[max(J0 - 2, 0):min(J1 + 2, nyl2), max(I0 - 2, 0):min(I1 + 2, nxl2)]
        bad += int((~win).sum())
    return bad


def test_proper_nesting_through_a_run_with_regrids():
    """The 3-level shelf (uplift, coast): after every coarse step each level-3
    patch keeps a 2-cell margin of level-2 cells around it."""
    w = W.amr3(L=240e3, dx1=4000.0, steps=16)
    cfg = dict(w["cfg"], regrid_interval=2)
    o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
    r1, r2 = cfg["ratios"]
    nxl2, nyl2 = cfg["nx"] * r1, cfg["ny"] * r1
    seen3 = 0
    for _ in range(16):
        o.step(1)
        seen3 += o.num_patches(0, 3)
        assert _nesting_violations(o, nxl2, nyl2, r2) == 0
    assert seen3 > 0


# --------------------------------------------------------------------------
# gauges

def _dry_hill(bed_fn, gauges, nx=32, dx=1000.0, r=4, region=None):
    """Dry land everywhere (B > 0, still sea at 0): nothing moves, and a gauge
    reads h + B = B, which every level samples from the topography at its own
    cell centres.  The topography grid has nodes at dx / 16, finer than level 2."""
    L = nx * dx
    n_in = 16 * nx + 1
    xs = np.linspace(0.0, L, n_in)
    X, Y = np.meshgrid(xs, xs)
    cfg = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_EXTRAP] * 4, dt_max=1.0,
                        num_levels=2 if region else 1, ratios=[r] if region else [],
                        regions=[region] if region else [], regrid_interval=0)
    w = dict(cfg=cfg, topo=[(bed_fn(X, Y), 0.0, 0.0, L / (n_in - 1), L / (n_in - 1))], eta=[], uplift=[],
             gauges=np.asarray(gauges, float))
    o = W.load(oracle.Oracle(cfg), w)
    if region:
        assert o.num_patches(0, 2) > 0
    o.step(2)
    assert np.abs(o.level_array(0, 1, "h")).max() == 0.0
    _, e = o.read_gauges()
    return e[-1].ravel()


def test_gauge_reads_a_linear_surface_exactly():
    """Bilinear interpolation between cell centres is exact on a plane."""
    s1, s2, L = 2e-4, -3e-4, 32e3
    fn = lambda x, y: 20.0 + s1 * (x - L / 2) + s2 * (y - L / 2)
    g = [[10400.0, 17700.0], [5000.0, 5000.0], [21234.5, 9876.5], [16000.0, 16250.0]]
    got = _dry_hill(fn, g)
    want = np.array([fn(x, y) for x, y in g])
    assert np.abs(got - want).max() <= 1e-11


def test_gauge_reads_the_finest_level():
    """B = 5 + q ((x - xc)^2 + (y - yc)^2) read at a corner of level-1 cells:
    bilinear interpolation between the four centres around it overshoots by
    q (dx^2 + dy^2) / 4 on the level read, so by 2 q dx1^2 / 4 on level 1 and
    by 16 times less on level 2 (ratio 4)."""
    q, L, dx, r = 1e-7, 32e3, 1000.0, 4
    fn = lambda x, y: 5.0 + q * ((x - L / 2) ** 2 + (y - L / 2) ** 2)
    g = [[14000.0, 15000.0], [17000.0, 16000.0]]          # level-1 cell corners inside the refined region
    region = [11000.0, 11000.0, 21000.0, 21000.0, 2, 2]
    want = np.array([fn(x, y) for x, y in g])
    fine = _dry_hill(fn, g, r=r, region=region) - want
    coarse = _dry_hill(fn, g) - want
    b1, b2 = q * 2 * dx ** 2 / 4, q * 2 * (dx / r) ** 2 / 4
    assert np.allclose(coarse, b1, rtol=1e-3)
    assert np.allclose(fine, b2, rtol=1e-2)


# --------------------------------------------------------------------------
# seafloor uplift

def _uplift_runs(when):
    """A 2-level basin with a beach and dry land, with no uplift and with a
    planar uplift dB = 0.5 + 2e-5 x - 1e-5 y (bilinear sampling is exact on a
    plane), given before or after init.  Level 2 covers deep water only: a
    level made at t = 0 is interpolated from level 1 (the initial state is
    set on level 1), and next to dry cells the limited slopes (minmod, one-
    sided against a dry neighbour) do not carry a planar
    uplift through exactly."""
    nx, dx = 40, 500.0
    L = nx * dx
    xs = np.linspace(0.0, L, 81)
    X, Y = np.meshgrid(xs, xs)
    bed = np.minimum(-20.0 + 40.0 * X / L, 6.0)                 # beach rising out of the sea at x = L / 2
    cfg = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_WALL] * 4, num_levels=2, ratios=[4],
                        regrid_interval=0, regions=[[0.1 * L, 0.2 * L, 0.4 * L, 0.7 * L, 2, 2]])
    w = dict(cfg=cfg, topo=[(bed, 0.0, 0.0, L / 80, L / 80)], eta=[], uplift=[], gauges=np.zeros((0, 2)))
    dB = 0.5 + 2e-5 * X - 1e-5 * Y
    up = (0, dB, 0.0, 0.0, L / 80, L / 80)
    o = oracle.Oracle(cfg)
    if when == "before":
        W.load(o, dict(w, uplift=[up]))
    else:
        W.load(o, w)
        if when == "after":
            o.add_uplift(*up)
    return o, cfg


def _levels(o):
    return {lev: o.patches(0, lev) for lev in (1, 2)}


@pytest.mark.parametrize("when", ["before", "after"])
def test_uplift_moves_bed_and_surface_together(when):
    """Sec. 5.1.1: the seafloor deformation is applied instantaneously, the
    water column moving with it: on every level B rises by dB at each cell
    centre, h and the mass stay, so eta rises by dB where wet and dry land
    stays dry."""
    ref, cfg = _uplift_runs("none")
    got, _ = _uplift_runs(when)
    assert abs(got.stats()["mass"] - ref.stats()["mass"]) <= 1e-14 * ref.stats()["mass"]
    a, b = _levels(ref), _levels(got)
    wet_seen = dry_seen = 0
    for lev in (1, 2):
        assert [p[0] for p in a[lev]] == [p[0] for p in b[lev]]
        d = cfg["dx"] / (4 ** (lev - 1))
        for (box, pa), (_, pb) in zip(a[lev], b[lev]):
            i0, j0, nx, ny = box
            X, Y = np.meshgrid((i0 + np.arange(nx) + 0.5) * d, (j0 + np.arange(ny) + 0.5) * d)
            dB = 0.5 + 2e-5 * X - 1e-5 * Y
            assert np.abs((pb["B"] - pa["B"]) - dB).max() <= 1e-12
            if lev == 1:
                assert np.array_equal(pb["h"], pa["h"])       # sampled directly
            else:
                assert np.abs(pb["h"] - pa["h"]).max() <= 1e-12  # interpolated from level 1
            wet = pa["h"] > 0
            eta_a, eta_b = pa["h"] + pa["B"], pb["h"] + pb["B"]
            assert np.abs((eta_b - eta_a)[wet] - dB[wet]).max() <= 1e-12
            if lev == 1:
                wet_seen += int(wet.sum())
                dry_seen += int((~wet).sum())
    assert wet_seen > 0 and dry_seen > 0


# --------------------------------------------------------------------------
# the zeta output field

def test_zeta_of_a_raised_still_sea_over_a_beach():
    """Sec. 5.1.2, Eq. (zeta): zeta is the surface offshore (B <= 0) and the
    water depth on land (B > 0).  A still sea at +0.5 m over a beach rising
    through sea level (any constant level is at rest) gives the closed form
    zeta = 0.5 offshore, 0.5 - B on flooded land (0 < B < 0.5), 0 above."""
    nx, dx = 64, 10.0
    L = nx * dx
    xs = np.linspace(0.0, L, 2 * nx + 1)
    X, _ = np.meshgrid(xs, np.linspace(0.0, 8 * dx, 17))
    bed = -2.0 + 4.0 * X / L                                  # B from -2 to +2 m: sea level at x = L / 2
    cfg = W.base_config(nx=nx, ny=8, dx=dx, dy=dx, bc=[W.BC_WALL] * 4)
    w = dict(cfg=cfg, topo=[(bed, 0.0, 0.0, L / (2 * nx), dx / 2)], eta=[(0, np.full((2, 2), 0.5), 0.0, 0.0, L, 8 * dx)],
             uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    o.step(10)
    xc = (np.arange(nx) + 0.5) * dx
    B = -2.0 + 4.0 * xc / L
    want = np.where(B <= 0.0, 0.5, np.maximum(0.5 - B, 0.0))
    zeta = o.read_field(0, 1, "zeta", nx, 1, xc[0], 4 * dx + 0.5 * dx, dx, dx)[0]
    assert np.abs(zeta - want).max() <= 1e-12
    assert (B > 0.5).any() and ((B > 0.0) & (B < 0.5)).any()   # dry land and flooded land both present
