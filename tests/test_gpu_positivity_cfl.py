"""GPU parity of the non-negative-depth bound of the Riemann solver and of the
CFL retake (Sec. 2.2), through the C ABI against the FP64 oracle.

Bars (as in test_gpu_parity.py): FP64 bit for bit, the time-step sequence and
the retake and violation counts included; FP32 perturbation form within
1e-4 m in surface elevation.  Also: a state that is not a finite number makes
tsu_step return TSU_ERR_NAN (the NaN is put in by the host, in the initial
velocity; no kernel is made to fault).
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
