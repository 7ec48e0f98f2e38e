"""GPU parity of the non-negative-depth bound of the Riemann solver and of the
CFL retake (Sec. 2.2), through the C ABI against the FP64 oracle.

Bars (as in test_gpu_parity.py): FP64 bit for bit, the time-step sequence and
the retake and violation counts included; FP32 perturbation form within
1e-4 m in surface elevation.  Also: a state that is not a finite number makes
tsu_step return TSU_ERR_NAN (the NaN is put in by the host, in the initial
velocity; no kernel is made to fault), and a kernel wait that runs out of its
poll budget makes it return TSU_ERR_TIMEOUT, and a negative depth written into
the state by the caller makes it return TSU_ERR_NEGDEPTH without stepping.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(cfg, precision=0, use_graphs=True):
    from paper_1901_06798_gb300 import binding
    return binding.Tsunami(cfg, precision=precision, use_graphs=use_graphs)


def _same_fields(o, g, nlev=1):
    for lev in range(1, nlev + 1):
        ob = [p[0] for p in o.patches(0, lev)]
        gb = [tuple(int(v) for v in b) for b in g.boxes(0, lev)]
        assert ob == gb, lev
        for (box, a), (_, b) in zip(o.patches(0, lev), g.patches(0, lev)):
            for f in ("h", "hu", "hv"):
                assert np.array_equal(a[f], b[f]), (lev, box, f, np.abs(a[f] - b[f]).max())


@pytest.mark.parametrize("seed", range(6))
def test_stepped_channels_f64_bitwise_with_dt_sequence(seed):
    """Random stepped channels: the depth bound changes these runs by 0.16 to
    0.82 m against a continuous-surface solver, and level-1 steps are retaken
    2 to 6 times in 30 steps.  One step per call (graph replay per parity), then
    a 10-step call (two-step graphs with the retake launches inside)."""
    w = W.stepped_channel(seed)
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g = W.load(_gpu(w["cfg"], 0), w)
    for _ in range(20):
        assert np.array_equal(o.step(1), g.step(1, allow_cfl=True))
    assert np.array_equal(o.step(10), g.step(10, allow_cfl=True))
    _same_fields(o, g)
    so, sg = o.stats(), g.stats()
    assert so["cfl_retakes"] == sg["cfl_retakes"] and so["cfl_retakes"] >= 1
    assert so["cfl_violations"] == sg["cfl_violations"]
    assert so["cell_updates"] == sg["cell_updates"]


def test_beach_runup_retakes_match_oracle_both_precisions():
    """A 1 m wave running up a dry beach retakes level-1 steps during the
    run-up: FP64 bit for bit with the same dt sequence and retake count.  In
    FP32 the thin films' speeds, u = hu / h with h near the dry tolerance,
    carry relative errors near 1e-4, and so does dt: the time stays within
    1e-4 relative of the oracle's and the FP32 run retakes too."""
    w = W.beach_runup()
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g = W.load(_gpu(w["cfg"], 0), w)
    g32 = W.load(_gpu(w["cfg"], 1), w)
    for _ in range(w["steps"]):
        to = o.step(1)
        assert np.array_equal(to, g.step(1))
        np.testing.assert_allclose(g32.step(1), to, rtol=1e-4)
    _same_fields(o, g)
    so = o.stats()
    assert so["cfl_retakes"] >= 2 and so["cfl_violations"] == 0
    assert g.stats()["cfl_retakes"] == so["cfl_retakes"]
    s32 = g32.stats()
    assert s32["cfl_retakes"] >= 1 and s32["cfl_violations"] == 0
    eo, e32 = o.level_array(0, 1, "eta"), g32.level_array(0, 1, "eta")
    wet = o.level_array(0, 1, "h") > 1e-3
    print(f"\nbeach run-up FP32: retakes {s32['cfl_retakes']} (oracle {so['cfl_retakes']}), "
          f"surface error {np.abs(e32 - eo)[wet].max():.2e} m, offshore {np.abs(e32 - eo)[:, :20].max():.2e} m")


def test_beach_runup_two_levels_f64_bitwise():
    """The same run-up under a ratio-4 level that follows the wave: the
    level-1 retakes happen with a finer level present (the finer level then
    steps with the retaken dt), and the finer level's own violations are kept
    and counted, the same on both sides."""
    w = W.beach_runup()
    cfg = dict(w["cfg"], num_levels=2, ratios=[4], regrid_interval=4, flag_eta_tol=0.05, patch_max=32)
    w = dict(w, cfg=cfg)
    o = W.load(oracle.Oracle(cfg), w)
    g = W.load(_gpu(cfg, 0), w)
    for _ in range(w["steps"]):
        assert np.array_equal(o.step(1), g.step(1, allow_cfl=True))
    _same_fields(o, g, nlev=2)
    so, sg = o.stats(), g.stats()
    assert so["cfl_retakes"] == sg["cfl_retakes"] >= 1
    assert so["cfl_violations"] == sg["cfl_violations"]
    assert so["cell_updates"] == sg["cell_updates"]


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_state_returns_tsu_err_nan(prec):
    """A NaN velocity in one wet cell (set by the host) makes the momentum NaN;
    within two steps the surface is NaN too, and tsu_step returns TSU_ERR_NAN
    instead of carrying on; later calls keep returning it."""
    from paper_1901_06798_gb300 import binding
    w = W.hump200()
    cfg = dict(w["cfg"], nx=64, ny=48)
    u = np.zeros((49, 65))
    u[20, 30] = np.nan
    w = dict(w, cfg=cfg, uv=[(0, u, np.zeros_like(u), 0.0, 0.0, 10.0, 10.0)])
    g = W.load(_gpu(cfg, prec), w)
    with pytest.raises(binding.TsuError) as e:
        g.step(3)
    assert e.value.code == binding.TSU_ERR_NAN
    with pytest.raises(binding.TsuError) as e:
        g.step(1)
    assert e.value.code == binding.TSU_ERR_NAN


@pytest.mark.parametrize("spherical", [False, True])
def test_bulk_row_copies_same_bits_as_per_thread_copies(spherical):
    """The x-sweep kernel's rows by bulk copies on mbarriers (tsu_set_bulk_copies)
    give the bits of the per-thread cp.async copies, on a Cartesian shelf with
    dry land and on the latitude-longitude grid, in the AMR levels too."""
    if spherical:
        # a hump running up a sloping beach between walls at 40 N, 2 degrees square
        n, box, x0, y0 = 48, 2.0, 200.0, 39.0
        d = box / n
        cfg = W.base_config(nx=n, ny=n, x0=x0, y0=y0, dx=d, dy=d, bc=[W.BC_WALL] * 4, spherical=1)
        X, Y = np.meshgrid(np.linspace(x0, x0 + box, n + 1), np.linspace(y0, y0 + box, n + 1))
        B = -60.0 + 75.0 * (X - x0) / box + 10.0 * np.sin(3.0 * (Y - y0))
        eta = W.gaussian_grid(x0, y0, box, box, n + 1, n + 1, x0 + 0.65 * box, 40.2, 2.0, 0.15, 0.2)[0]
        w = dict(cfg=cfg, topo=[(B, x0, y0, d, d)], eta=[(0, eta, x0, y0, d, d)], uplift=[], gauges=np.zeros((0, 2)))
    else:
        w = W.shelf(n=96, dx=2000.0)
    cfg = dict(w["cfg"], num_levels=2, ratios=[4], regrid_interval=3, flag_eta_tol=0.05, patch_max=32)
    w = dict(w, cfg=cfg)
    ref = W.load(_gpu(cfg, 1), w)
    blk = W.load(_gpu(cfg, 1), w)
    blk.set_bulk_copies(1)
    assert np.array_equal(ref.step(6), blk.step(6))
    for lev in (1, 2):
        for (b0, a), (b1, b) in zip(ref.patches(0, lev), blk.patches(0, lev)):
            assert np.array_equal(b0, b1)
            for f in ("h", "hu", "hv"):
                assert np.array_equal(a[f], b[f]), (lev, f)


def test_wait_budget_zero_returns_tsu_err_timeout():
    """With bulk row copies and a poll budget of 0 the x-sweep kernel's first
    wait gives up: the work item issues no further copies, waits for those in
    flight, and the step returns TSU_ERR_TIMEOUT; later calls keep returning
    it (no GPU fault is involved).  A context with the default budget steps
    the same workload to the oracle's time; bad arguments are TSU_ERR_ARG."""
    from paper_1901_06798_gb300 import binding
    w = W.hump200()
    g = W.load(_gpu(w["cfg"], 1), w)
    for en, polls in ((2, 10), (1, -1), (1, 1 << 32)):
        with pytest.raises(binding.TsuError) as e:
            g.set_bulk_copies(en, polls)
        assert e.value.code == binding.TSU_ERR_ARG
    g.set_bulk_copies(1, 0)
    for _ in range(2):
        with pytest.raises(binding.TsuError) as e:
            g.step(1)
        assert e.value.code == binding.TSU_ERR_TIMEOUT
    o = W.load(oracle.Oracle(w["cfg"]), w)
    g2 = W.load(_gpu(w["cfg"], 1), w)
    g2.set_bulk_copies(1)
    np.testing.assert_allclose(g2.step(3), o.step(3), rtol=1e-5)


def _cudart():
    import ctypes
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("no CUDA runtime library to copy through")


@pytest.mark.parametrize("prec", [0, 1])
def test_negative_depth_written_by_the_caller_returns_tsu_err_negdepth(prec):
    """A negative depth written into the level-1 state through
    tsu_level1_buffers (by the host, with cudaMemcpy) makes the next tsu_step
    return TSU_ERR_NEGDEPTH without stepping, and every step after it until
    the state is repaired; then the run continues to the oracle's time."""
    import ctypes
    from paper_1901_06798_gb300 import binding
    rt = _cudart()
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    w = W.hump200()
    g = W.load(_gpu(w["cfg"], prec), w)
    (ph, _, _, pB), pitch = g.level1_buffers()
    dt = np.float64 if prec == 0 else np.float32
    off = ((20 + 2) * pitch + 30 + 2) * np.dtype(dt).itemsize
    old, B = np.zeros(1, dt), np.zeros(1, dt)
    assert rt.cudaMemcpy(old.ctypes.data, ph + off, old.nbytes, 2) == 0     # device to host
    assert rt.cudaMemcpy(B.ctypes.data, pB + off, B.nbytes, 2) == 0
    bad = np.array([-0.25 if prec == 0 else B[0] - 0.25], dt)
    assert rt.cudaMemcpy(ph + off, bad.ctypes.data, bad.nbytes, 1) == 0     # host to device
    for _ in range(2):
        with pytest.raises(binding.TsuError) as e:
            g.step(1)
        assert e.value.code == binding.TSU_ERR_NEGDEPTH
    assert g.stats()["t"] == 0.0
    assert rt.cudaMemcpy(ph + off, old.ctypes.data, old.nbytes, 1) == 0
    o = W.load(oracle.Oracle(w["cfg"]), w)
    np.testing.assert_allclose(g.step(2), o.step(2), rtol=1e-5)
