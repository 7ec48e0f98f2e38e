"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bars (written here; FP32 rounding in the perturbation form is 1e-7 m per step on O(1 m) values):
  * FP64: relative error per field (max |gpu - oracle| / max |oracle|) <= 1e-12
    after the stated steps; patch lists (integer work) bit-exact; the FP64
    kernels are built without contraction and follow the oracle's operation
    order, so most cases are checked bit for bit as well.
  * FP32 perturbation form: surface elevation within 1e-4 m of the oracle,
    per field and per gauge.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64_REL = 1e-12
F32P_ETA = 1e-4


def _gpu(cfg, precision=0, use_graphs=True):
    from paper_1901_06798_gb300 import binding
    return binding.Tsunami(cfg, precision=precision, use_graphs=use_graphs)


def run_pair(w, steps, precision=0, use_graphs=True, cfg=None):
    cfg = cfg or w["cfg"]
    w = dict(w, cfg=cfg)
    o = W.load(oracle.Oracle(cfg), w)
    g = W.load(_gpu(cfg, precision, use_graphs), w)
    if steps:
        o.step(steps)
        g.step(steps)
    return o, g


def rel_err(a, b):
    m = np.nanmax(np.abs(b))
    return np.nanmax(np.abs(a - b)) / (m if m > 0 else 1.0)


def compare_levels(o, g, nlev, nscen=1, bitwise=False, tol=F64_REL):
    for s in range(nscen):
        for lev in range(1, nlev + 1):
            ob = [p[0] for p in o.patches(s, lev)]
            gb = [tuple(int(v) for v in b) for b in g.boxes(s, lev)]
            assert ob == gb, f"patch lists differ on level {lev} scenario {s}"
            for (box, a), (_, b) in zip(o.patches(s, lev), g.patches(s, lev)):
                for f in ("h", "hu", "hv", "B"):
                    if bitwise:
                        assert np.array_equal(a[f], b[f]), (lev, box, f, np.abs(a[f] - b[f]).max())
                    else:
                        assert rel_err(b[f], a[f]) <= tol, (lev, box, f, rel_err(b[f], a[f]))


def test_hump200_f64_matches_oracle():
    w = W.hump200()
    o, g = run_pair(w, 100)
    compare_levels(o, g, 1)
    so, sg = o.stats(), g.stats()
    assert so["dt"] == sg["dt"] and so["t"] == sg["t"]
    assert sg["cell_updates"] == 4.0e6


def test_hump200_f64_bitwise():
    w = W.hump200()
    o, g = run_pair(w, 100)
    compare_levels(o, g, 1, bitwise=True)


def test_ragged_tiles_and_strips():
    """Uneven tiles (37) and widths that leave ragged strips and segments."""
    w = W.hump200()
    cfg = dict(w["cfg"], level1_tile=37)
    o, g = run_pair(w, 40, cfg=cfg)
    assert g.num_patches(0, 1) == 36
    compare_levels(o, g, 1, bitwise=True)
    cfg = dict(w["cfg"], nx=133, ny=71, level1_tile=0)
    o, g = run_pair(dict(w, cfg=cfg), 25, cfg=cfg)
    compare_levels(o, g, 1, bitwise=True)


def test_tiny_grid_and_single_column_patches():
    w = W.hump200()
    cfg = dict(w["cfg"], nx=5, ny=3, dx=400.0, dy=400.0, level1_tile=2)
    o, g = run_pair(dict(w, cfg=cfg), 10, cfg=cfg)
    compare_levels(o, g, 1, bitwise=True)


def test_more_patches_than_a_grid_y_extent():
    """70,225 patches on one level (2 x 2 tiles of a 530^2 shelf with beach and
    dry land), more than the 65,535 rows a CUDA grid's y extent allows: the
    patch-batched kernels (ghost fill, boundaries, field reads, mass) index the
    patch by blockIdx.x.  The tiled level steps to the same bits as one patch
    in FP64; in the FP32 perturbation form it stays within 1e-5 m of it."""
    from paper_1901_06798_gb300 import binding
    w = W.shelf(n=530, dx=2000.0, steps=20)
    tiled = dict(w["cfg"], level1_tile=2)
    pts = (530, 530, 1000.0, 1000.0, 2000.0, 2000.0)
    for prec in (binding.TSU_F64, binding.TSU_F32P):
        one = W.load(_gpu(w["cfg"], prec), w)
        many = W.load(_gpu(tiled, prec), dict(w, cfg=tiled))
        assert many.num_patches(0, 1) == 265 * 265
        one.step(20)
        many.step(20)
        t1, t2 = one.stats()["t"], many.stats()["t"]
        assert t1 == t2 if prec == binding.TSU_F64 else abs(t1 - t2) <= 1e-6 * t1
        got = {}
        for f in ("eta", "hu", "hv"):
            a = one.read_field(0, 1, f, *pts)
            got[f] = many.read_field(0, 1, f, *pts)
            assert not np.isnan(got[f]).any()
            if prec == binding.TSU_F64:
                assert np.array_equal(a, got[f]), f
            else:
                assert np.abs(a - got[f]).max() <= 1e-5, (f, np.abs(a - got[f]).max())
        # a field of more than 8 MiB takes the read-back path for large fields:
        # four points per cell, piecewise constant
        big = many.read_field(0, 1, "eta", 1060, 1060, 500.0, 500.0, 1000.0, 1000.0)
        assert np.array_equal(big[::2, ::2], got["eta"]) and np.array_equal(big[1::2, 1::2], got["eta"])
        if prec == binding.TSU_F64:
            # the same cells summed in another order (per patch, then patch by patch)
            assert abs(one.stats()["mass"] - many.stats()["mass"]) <= 1e-10 * abs(one.stats()["mass"])
        one.close()
        many.close()


@pytest.mark.parametrize("retake", [0, 1])
def test_timed_steps_are_the_steps_tsu_step_takes(retake):
    """The bench times steps with tsu_time_level1_steps: they must be the steps
    tsu_step takes (the same kernels, the CFL retake pass included when it is
    on), so both contexts end with the same bits and the same time."""
    w = W.shelf(n=192, dx=2000.0, steps=12)
    cfg = dict(w["cfg"], cfl_retake=retake)
    a = W.load(_gpu(cfg, 1, use_graphs=False), dict(w, cfg=cfg))
    b = W.load(_gpu(cfg, 1), dict(w, cfg=cfg))
    km, sm = a.time_level1_steps(2, 10)
    assert 0.0 < km <= sm
    b.step(12)
    assert a.stats()["t"] == b.stats()["t"] and a.stats()["dt"] == b.stats()["dt"]
    for f in ("eta", "hu", "hv"):
        assert np.array_equal(a.level_array(0, 1, f), b.level_array(0, 1, f)), f


def test_shelf_with_dry_land_f64():
    w = W.shelf(n=192, dx=2000.0, steps=60)
    o, g = run_pair(w, 60)
    compare_levels(o, g, 1, bitwise=True)


def test_lake_at_rest_gpu_both_precisions():
    """Still sea with beach and dry land: exactly at rest after 1000 steps."""
    w = W.lake_at_rest_shelf(n=96)
    for prec in (0, 1):
        g = W.load(_gpu(w["cfg"], prec), w)
        g.step(1000)
        for f in ("hu", "hv"):
            assert np.abs(g.level_array(0, 1, f)).max() == 0.0
        eta = g.read_field(0, 1, "eta", 96, 96, 1000.0, 1000.0, 2000.0, 2000.0)
        h = g.read_field(0, 1, "h", 96, 96, 1000.0, 1000.0, 2000.0, 2000.0)
        assert np.abs(eta[h > 0]).max() == 0.0


@pytest.mark.parametrize("name,steps", [("hump", 100), ("shelf", 100), ("shelf", 500)])
def test_f32_perturbation_within_1e4_m(name, steps):
    """FP32 perturbation form against the FP64 oracle; the 500-step shelf run
    is the bench workload's step count on a 192^2 grid with the same bed
    profile, uplift, beach and dry land."""
    w = W.hump200() if name == "hump" else W.shelf(n=192, dx=2000.0, steps=steps)
    o, g = run_pair(w, steps, precision=1)
    e_o = o.level_array(0, 1, "eta")
    e_g = g.level_array(0, 1, "eta")
    wet = o.level_array(0, 1, "h") > 0
    err = np.abs(e_g - e_o)[wet].max()
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    gerr = np.abs(eg - eo).max()
    print(f"\n{name} {steps} steps: max |eta - eta_oracle| {err:.3e} m (wet cells), gauges {gerr:.3e} m, "
          f"max |eta| {np.abs(e_o[wet]).max():.3f} m")
    assert err <= F32P_ETA
    assert gerr <= F32P_ETA
    assert np.allclose(tg, to, rtol=1e-5)


def test_graph_replay_equals_eager():
    w = W.shelf(n=128, dx=2000.0)
    a = W.load(_gpu(w["cfg"], 0, use_graphs=True), w)
    b = W.load(_gpu(w["cfg"], 0, use_graphs=False), w)
    a.step(9)
    b.step(9)
    for f in ("h", "hu", "hv"):
        assert np.array_equal(a.level_array(0, 1, f), b.level_array(0, 1, f))
    ta, ea = a.read_gauges()
    tb, eb = b.read_gauges()
    assert np.array_equal(ta, tb) and np.array_equal(ea, eb)


@pytest.mark.parametrize("prec", [0, 1])
def test_single_step_graphs_equal_eager(prec):
    """Single-step calls replay one graph per buffer-parity pattern; they must
    give the eager run bit for bit, on a tiled level and under AMR whose
    regrids come every 4 coarse steps (graphs between regrids, eager around
    them), with every step's returned time equal."""
    w = W.shelf(n=128, dx=2000.0)
    cfg = dict(w["cfg"], level1_tile=40)
    wa = W.amr3(L=240e3, dx1=4000.0, steps=6)
    cfga = dict(wa["cfg"], regrid_interval=16)
    for ww, c, nlev, steps in ((w, cfg, 1, 7), (wa, cfga, 3, 13)):
        a = W.load(_gpu(c, prec, use_graphs=True), dict(ww, cfg=c))
        b = W.load(_gpu(c, prec, use_graphs=False), dict(ww, cfg=c))
        for _ in range(steps):
            assert np.array_equal(a.step(1), b.step(1))
        compare_levels(a, b, nlev, bitwise=True)
        ta, ea = a.read_gauges()
        tb, eb = b.read_gauges()
        assert np.array_equal(ta, tb) and np.array_equal(ea, eb)
        assert a.stats()["cell_updates"] == b.stats()["cell_updates"]
    assert a.num_patches(0, 3) > 0


def test_mixed_call_lengths_graphs_equal_eager():
    """Calls of different lengths mix one- and two-step graphs with eager
    steps; a single step changes level 1's buffer parity, so a two-step graph
    captured at one parity must not be replayed at the other.  The sequence
    2, 1, 2, 3, 2, 1, 1, 2 must give the eager run bit for bit (FP64), every
    returned time included, on a tiled level and under 3-level AMR."""
    w = W.shelf(n=128, dx=2000.0)
    cfg = dict(w["cfg"], level1_tile=40)
    wa = W.amr3(L=240e3, dx1=4000.0, steps=6)
    cfga = dict(wa["cfg"], regrid_interval=16)
    seq = (2, 1, 2, 3, 2, 1, 1, 2)
    for ww, c, nlev in ((w, cfg, 1), (wa, cfga, 3)):
        a = W.load(_gpu(c, 0, use_graphs=True), dict(ww, cfg=c))
        b = W.load(_gpu(c, 0, use_graphs=False), dict(ww, cfg=c))
        for n in seq:
            assert np.array_equal(a.step(n), b.step(n))
        compare_levels(a, b, nlev, bitwise=True)
        ta, ea = a.read_gauges()
        tb, eb = b.read_gauges()
        assert np.array_equal(ta, tb) and np.array_equal(ea, eb)
        assert a.stats()["cell_updates"] == b.stats()["cell_updates"]


def test_step_level_in_recursion_order_equals_tsu_step():
    """tsu_step_level driven in the order of the recursion of Sec. 3.1 (a
    level-1 step, then r substeps of level 2, each followed by its r substeps
    of level 3) gives tsu_step's run bit for bit over 6 coarse steps with
    regrids; calls out of that order return TSU_ERR_ARG and change nothing."""
    from paper_1901_06798_gb300 import binding
    w = _amr_small()
    cfg = w["cfg"]
    a = W.load(_gpu(cfg, 0), w)
    b = W.load(_gpu(cfg, 0, use_graphs=False), w)
    nlev, ratios = cfg["num_levels"], cfg["ratios"]

    def drive(g, lev):
        g.step_level(lev, allow_cfl=True)
        if lev < nlev and g.num_patches(0, lev + 1) > 0:
            for _ in range(ratios[lev - 1]):
                drive(g, lev + 1)

    for _ in range(6):
        drive(a, 1)
        b.step(1, allow_cfl=True)
    assert a.num_patches(0, 3) > 0
    compare_levels(a, b, 3, bitwise=True)
    ta, ea = a.read_gauges()
    tb, eb = b.read_gauges()
    assert np.array_equal(ta, tb) and np.array_equal(ea, eb)
    sa, sb = a.stats(), b.stats()
    assert sa["cell_updates"] == sb["cell_updates"] and sa["t"] == sb["t"]
    for bad in (lambda: a.step_level(2), lambda: a.step_level(0), lambda: a.step_level(4)):
        with pytest.raises(binding.TsuError) as e:
            bad()
        assert e.value.code == binding.TSU_ERR_ARG
    a.step_level(1, allow_cfl=True)   # level 2's substeps are now pending
    for bad in (lambda: a.step(1), lambda: a.step_level(1), lambda: a.step_level(3)):
        with pytest.raises(binding.TsuError) as e:
            bad()
        assert e.value.code == binding.TSU_ERR_ARG


def test_autotune_leaves_the_solution_unchanged():
    """The autotuner times zero-length steps: afterwards the run still matches
    the oracle bit for bit, in whatever launch shape it chose."""
    w = W.shelf(n=192, dx=2000.0)
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g = W.load(_gpu(w["cfg"], 0), w)
    o.step(3)
    g.step(3)
    nt, seg, ms = g.autotune(2)
    assert nt in (64, 128, 256) and seg in (32, 64, 128, 256) and ms > 0
    o.step(5)
    g.step(5)
    compare_levels(o, g, 1, bitwise=True)
    g32 = W.load(_gpu(w["cfg"], 1), w)
    g32.autotune(2)
    g32.step(8)
    assert np.abs(g32.level_array(0, 1, "eta") - o.level_array(0, 1, "eta")).max() <= F32P_ETA


def _amr_small():
    w = W.amr3(L=240e3, dx1=4000.0, steps=6)
    return w


def test_amr3_f64_patch_lists_fields_and_gauges():
    w = _amr_small()
    o, g = run_pair(w, 6)
    assert o.num_patches(0, 3) > 0
    compare_levels(o, g, 3, bitwise=True)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(to, tg)
    assert np.array_equal(eo, eg)
    so, sg = o.stats(), g.stats()
    assert so["cell_updates"] == sg["cell_updates"]
    # finest-level field sampling
    L = w["cfg"]["nx"] * w["cfg"]["dx"]
    fo = o.read_field(0, 0, "zeta", 97, 89, 100.0, 50.0, L / 97, L / 89)
    fg = g.read_field(0, 0, "zeta", 97, 89, 100.0, 50.0, L / 97, L / 89)
    assert np.array_equal(np.isnan(fo), np.isnan(fg))
    assert np.array_equal(fo[~np.isnan(fo)], fg[~np.isnan(fg)])


def test_amr3_f32p_gauges_within_1e4_m():
    w = _amr_small()
    o, g = run_pair(w, 6, precision=1)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.abs(eg - eo).max() <= F32P_ETA


def test_amr_lake_at_rest_gpu():
    """Still sea under 3-level AMR, regridding every 2 steps: exactly at rest on
    every level after 63 coarse steps (1008 steps of the finest level)."""
    w = W.amr3(L=120e3, dx1=4000.0, steps=6)
    cfg = dict(w["cfg"], regrid_interval=2)
    w = dict(w, cfg=cfg, uplift=[])
    for prec in (0, 1):
        g = W.load(_gpu(cfg, prec), w)
        assert g.num_patches(0, 3) > 0
        g.step(63)
        assert g.num_patches(0, 3) > 0
        for lev in (1, 2, 3):
            for box, a in g.patches(0, lev):
                assert np.abs(a["hu"]).max() == 0.0 and np.abs(a["hv"]).max() == 0.0


def test_ensemble_scenarios_match_oracle():
    w = W.ensemble(n_scen=3, n=64, dx=8000.0, steps=6)
    o, g = run_pair(w, 6)
    compare_levels(o, g, 2, nscen=3, bitwise=True)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(eo, eg)


def test_empty_finer_level():
    """No cell is flagged: level 2 stays empty and level 1 still matches."""
    w = W.hump200()
    cfg = dict(w["cfg"], num_levels=2, ratios=[4], regrid_interval=2, flag_eta_tol=10.0)
    o, g = run_pair(dict(w, cfg=cfg), 8, cfg=cfg)
    assert g.num_patches(0, 2) == 0
    compare_levels(o, g, 2, bitwise=True)


def test_full_size_shelf4096_properties():
    """The 4096^2 uniform run in the benchmark's launch configuration: at rest
    it stays exactly at rest; with the uplift (symmetric about mid-y) the
    solution stays mirror-symmetric in y; a window around the uplift matches
    the oracle run on a crop holding the whole domain of dependence."""
    from paper_1901_06798_gb300 import binding
    w = W.shelf(n=4096, dx=500.0)
    for prec in (0, 1):
        g = W.load(_gpu(w["cfg"], prec), dict(w, uplift=[], gauges=np.zeros((0, 2))))
        g.step(4)
        b = g.boxes(0, 1)
        assert len(b) == 1
        pts = np.linspace(1000.0, 4096 * 500.0 - 1000.0, 256)
        hu = g.read_field(0, 1, "hu", 256, 256, pts[0], pts[0], pts[1] - pts[0], pts[1] - pts[0])
        assert np.abs(hu).max() == 0.0
        g.close()
    k = 3
    g = W.load(_gpu(w["cfg"], 0), dict(w, gauges=np.zeros((0, 2))))
    g.step(k)
    n, dx = 4096, 500.0
    # y-mirror symmetry of the full field (sampled on a symmetric set of rows)
    xs = 1024e3 - 600e3 + (np.arange(-300, 300) + 0.5) * dx + 1024e3 * 0.0
    xs = (2048e3 - 600e3) + (np.arange(-300, 300) + 0.5) * dx
    ys = 1024e3 + (np.arange(-400, 400) + 0.5) * dx
    eta = g.read_field(0, 1, "eta", len(xs), len(ys), xs[0], ys[0], dx, dx)
    assert np.abs(eta - eta[::-1, :]).max() <= 1e-12 * np.abs(eta).max()
    # oracle on a crop that contains the uplift and the domain of dependence
    ci0, cj0 = int(xs[0] / dx) - 4 * k - 8, int(ys[0] / dx) - 4 * k - 8
    cw, ch = len(xs) + 2 * (4 * k + 8), len(ys) + 2 * (4 * k + 8)
    ccfg = dict(w["cfg"], nx=cw, ny=ch, x0=ci0 * dx, y0=cj0 * dx)
    o = W.load(oracle.Oracle(ccfg), dict(w, cfg=ccfg, gauges=np.zeros((0, 2))))
    o.step(k)
    assert o.stats()["dt"] == g.stats()["dt"]
    eo = o.read_field(0, 1, "eta", len(xs), len(ys), xs[0], ys[0], dx, dx)
    assert rel_err(eta, eo) <= F64_REL


def test_amr4_bay_four_levels_ratio_8():
    """The 4-level bay workload scaled down (96 km, ratios 4, 4, 8, the
    finest level forced around the bay and capped elsewhere): FP64 patch
    lists, fields and gauges bit for bit; FP32 gauges within 1e-4 m."""
    w = W.amr4_bay(L=96e3, dx1=4000.0, radius=1200.0, box=3000.0)
    o, g = run_pair(w, 4)
    assert o.num_patches(0, 4) > 0
    compare_levels(o, g, 4, bitwise=True)
    to, eo = o.read_gauges()
    tg, eg = g.read_gauges()
    assert np.array_equal(eo, eg)
    o, g = run_pair(w, 4, precision=1)
    _, eo = o.read_gauges()
    _, eg = g.read_gauges()
    assert np.abs(eg - eo).max() <= F32P_ETA


def test_mass_is_reproducible():
    """tsu_get_stats sums the mass in FP64 in a fixed order: the same state
    gives the same bits, call after call and context after context, and it
    agrees with the oracle's mass."""
    w = _amr_small()
    o, g = run_pair(w, 6, precision=0)
    g2 = W.load(_gpu(w["cfg"], 0), w)
    g2.step(6)
    m = [g.stats()["mass"] for _ in range(3)] + [g2.stats()["mass"]]
    assert all(x == m[0] for x in m), m
    assert abs(m[0] - o.stats()["mass"]) <= 1e-12 * abs(o.stats()["mass"])


def _beach_basin():
    """A 2-level basin with a beach and dry land, level 2 over deep water."""
    nx, dx = 40, 500.0
    L = nx * dx
    xs = np.linspace(0.0, L, 81)
    X, Y = np.meshgrid(xs, xs)
    bed = np.minimum(-20.0 + 40.0 * X / L, 6.0)
    cfg = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_WALL] * 4, num_levels=2, ratios=[4],
                        regrid_interval=0, regions=[[0.1 * L, 0.2 * L, 0.4 * L, 0.7 * L, 2, 2]])
    w = dict(cfg=cfg, topo=[(bed, 0.0, 0.0, L / 80, L / 80)], eta=[], uplift=[], gauges=np.array([[4000.0, 9000.0]]))
    up = (0, 0.5 + 2e-5 * X - 1e-5 * Y + 0.3 * np.exp(-((X - 5000.0) ** 2 + (Y - 9000.0) ** 2) / 2e6),
          0.0, 0.0, L / 80, L / 80)
    return cfg, w, up


def test_uplift_after_init_matches_oracle():
    """A deformation given after init (the bed and the surface move together
    on every level) and then stepped: FP64 bit for bit with the oracle."""
    cfg, w, up = _beach_basin()
    o = W.load(oracle.Oracle(cfg), w)
    g = W.load(_gpu(cfg, 0), w)
    o.add_uplift(*up)
    g.add_uplift(*up)
    for lev in (1, 2):
        for (bo, a), (bg, b) in zip(o.patches(0, lev), g.patches(0, lev)):
            for f in ("h", "B"):
                assert np.array_equal(a[f], b[f]), (lev, f)
    o.step(8)
    g.step(8)
    for lev in (1, 2):
        for (bo, a), (bg, b) in zip(o.patches(0, lev), g.patches(0, lev)):
            for f in ("h", "hu", "hv"):
                assert np.array_equal(a[f], b[f]), (lev, f)
    assert np.array_equal(o.read_gauges()[1], g.read_gauges()[1])


def test_time_step_follows_the_fastest_level_gpu():
    """A trench only level 2 resolves sets the step: the same dt sequence as
    the oracle, bit for bit, starting at nu dx1 / sqrt(g 100)."""
    nx, dx, nu = 16, 1000.0, 0.9
    L = nx * dx
    xs = np.arange(0.0, L + 1.0, dx / 16)
    bed = np.tile(np.where((xs >= 1000.0) & (xs <= 1250.0), -100.0, -10.0), (17, 1))
    cfg = W.base_config(nx=nx, ny=nx, dx=dx, dy=dx, bc=[W.BC_WALL] * 4, num_levels=2, ratios=[4], cfl_desired=nu,
                        regrid_interval=0, regions=[[0.0, 0.0, 3000.0, L, 2, 2]])
    w = dict(cfg=cfg, topo=[(bed, 0.0, 0.0, dx / 16, L / 16)], eta=[], uplift=[], gauges=np.zeros((0, 2)))
    o = W.load(oracle.Oracle(cfg), w)
    g = W.load(_gpu(cfg, 0), w)
    to, tg = o.step(1)[0], g.step(1)[0]
    assert to == tg
    assert abs(tg - nu * dx / np.sqrt(9.81 * 100.0)) <= 1e-13 * tg
    for _ in range(10):
        assert o.step(1)[0] == g.step(1)[0]
    assert g.stats()["cfl_violations"] == 0
