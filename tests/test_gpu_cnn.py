"""The refinement-flag predictor on the GPU, through the C ABI:

* forward (FP32, and FP16 inference with FP32 accumulation), loss and
  gradient against the FP64 oracle of oracle/cnn.py;
* the feature planes of a level against their definition on the oracle's
  fields;
* training on the GPU on flags the method itself generates, and what the
  trained network gains over plain b-cell buffering: fewer cell updates, no
  missed flags, and gauges as close to a uniform fine-grid reference as with
  plain flagging.

Tolerances: FP32 forward 1e-4 and gradient 1e-4 of the largest entry (FP32
sums of <= 144 terms per output, three layers deep); FP16 inference 2e-2 of
the largest logit (inputs and weights rounded to 11-bit mantissas, u = 4.9e-4,
through three layers of 144-term sums) -- used only to threshold logits.
"""
import numpy as np
import pytest

import oracle
from oracle import cnn as ocnn
from paper_1901_06798_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rand_batch(seed, n=2, h=19, w=23):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, ocnn.C_IN, h, w))
    x[:, 4] = (rng.random((n, h, w)) < 0.3)
    t = (rng.random((n, h, w)) < 0.25).astype(float)
    m = (rng.random((n, h, w)) < 0.9).astype(float)
    return x, t, m


def test_forward_matches_oracle():
    from paper_1901_06798_gb300 import binding
    theta = ocnn.init_params(3)
    x, _, _ = _rand_batch(1)
    ref, _ = ocnn.forward(theta, x)
    out32 = binding.cnn_forward(theta, x, fp16=False)
    out16 = binding.cnn_forward(theta, x, fp16=True)
    scale = np.abs(ref).max()
    assert np.abs(out32 - ref).max() <= 1e-4 * scale
    assert np.abs(out16 - ref).max() <= 2e-2 * scale
    assert binding.cnn_num_params() == ocnn.n_params()


def test_loss_and_gradient_match_oracle():
    from paper_1901_06798_gb300 import binding
    theta = ocnn.init_params(4) * 0.8
    x, t, m = _rand_batch(2, n=3, h=17, w=21)
    loss_ref, g_ref = ocnn.backward(theta, x, t, m)
    loss, g = binding.cnn_loss_grad(theta, x, t, m)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_feature_planes_match_definition():
    from paper_1901_06798_gb300 import binding
    w = W.shelf(n=128, dx=4000.0)
    cfg = dict(w["cfg"], flag_eta_tol=0.02, flag_depth_below=200.0)
    o = W.load(oracle.Oracle(cfg), dict(w, cfg=cfg))
    g = W.load(binding.Tsunami(cfg, precision=0), dict(w, cfg=cfg))
    o.step(6)
    g.step(6)
    f, fl = g.cnn_features(0, 1)
    h, hu, hv, B = (o.level_array(0, 1, k) for k in ("h", "hu", "hv", "B"))
    crit = ((h >= cfg["drytol"]) & (np.abs(h + B) > cfg["flag_eta_tol"])) | (-B < cfg["flag_depth_below"])
    assert np.array_equal(fl.astype(bool), crit)
    ref = ocnn.features(h, hu, hv, B, np.ones_like(h, dtype=bool), crit)
    assert np.abs(f - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


def _ensemble_cfg(n_scen, use_cnn=0, b=4):
    w = W.ensemble(n_scen=n_scen, n=256, dx=4000.0, ratio=4, steps=0, seed=7)
    cfg = dict(w["cfg"], flag_eta_tol=0.02, regrid_interval=b, use_cnn=use_cnn, cnn_buffer=1, patch_max=64)
    return dict(w, cfg=cfg)


def _log_pairs(n_scen=6, regrids=16, b=4):
    """Features at each regrid and the criterion flags one regrid later."""
    from paper_1901_06798_gb300 import binding
    w = _ensemble_cfg(n_scen, b=b)
    g = W.load(binding.Tsunami(w["cfg"], precision=1), dict(w, gauges=np.zeros((0, 2))))
    X, T, prev = [], [], [None] * n_scen
    for _ in range(regrids):
        for s in range(n_scen):
            f, fl = g.cnn_features(s, 1)
            if prev[s] is not None:
                X.append(prev[s])
                T.append(fl.astype(np.float32))
            prev[s] = f
        g.step(b)
    return np.stack(X), np.stack(T)


def _cnn_vs_plain(theta, buffer):
    """One unseen uplift scenario over 40 coarse steps with plain b = 4 buffering
    and with the predictor (flags = criterion now, union prediction, dilated by
    `buffer`): cell updates, criterion-flagged cells left unrefined, wall time,
    and the largest gauge difference between the two runs at the plain run's
    times (each run chooses its own dt)."""
    import time
    from paper_1901_06798_gb300 import binding
    up = [(0, *W.shelf_uplift(1024e3, 1024e3, scale=0.5, amp=3.0, s_km=640.0, yc=540e3))]
    gauges = np.array([[674e3, 540e3], [744e3, 560e3], [774e3, 500e3]])
    runs = {}
    for name, use in (("plain", 0), ("cnn", 1)):
        w = dict(_ensemble_cfg(1, use_cnn=use), uplift=up)
        w = dict(w, cfg=dict(w["cfg"], cnn_buffer=buffer))
        c = binding.Tsunami(w["cfg"], precision=1)
        if use:
            c.cnn_set_weights(theta)
        W.load(c, dict(w, gauges=gauges))
        misses, wall = 0, 0.0
        for _ in range(40):
            c.sync()
            t0 = time.perf_counter()
            c.step(1)
            c.sync()
            wall += time.perf_counter() - t0
            _, fl = c.cnn_features(0, 1)
            cov = np.zeros_like(fl, dtype=bool)
            for (i0, j0, nx, ny) in c.boxes(0, 2):
                cov[j0 // 4:(j0 + ny) // 4, i0 // 4:(i0 + nx) // 4] = True
            misses += int(((fl > 0) & ~cov).sum())
        t, e = c.read_gauges()
        runs[name] = (c.stats()["cell_updates"], misses, t[:, 0], e[:, 0, :], wall)
    cu_p, mi_p, t_p, e_p, w_p = runs["plain"]
    cu_c, mi_c, t_c, e_c, w_c = runs["cnn"]
    n = min(len(t_p), len(t_c))
    e_ci = np.stack([np.interp(t_p[:n], t_c, e_c[:, k]) for k in range(gauges.shape[0])], axis=1)
    diff = float(np.abs(e_ci - e_p[:n]).max())
    print(f"\npredictor, buffer {buffer}: cell updates {cu_c / cu_p:.3f} of plain b = 4, step wall time "
          f"{w_c:.3f} s vs {w_p:.3f} s, gauges within {diff:.2e} m of plain (amplitude "
          f"{np.abs(e_p).max():.2f} m), misses {mi_c}")
    return cu_c / cu_p, mi_p, mi_c, diff


def test_trained_predictor_against_plain_buffering():
    """What the trained predictor buys over plain b = 4 buffering, judged by
    the criterion (no flagged cell left unrefined) and by the gauges.  With the
    predictor's cells dilated by 1 it refines fewer cells than plain
    buffering; dilated by 2 its gauges agree with plain buffering's within
    1e-4 m.  On this workload the two do not meet: at an equal gauge error the
    learned flags refine about 2% more cells, and the 2% fewer cells of buffer
    1 cost gauge differences of a few mm, because the plain buffer also keeps
    the wave's tail below the criterion refined (the numbers are printed)."""
    from paper_1901_06798_gb300 import binding
    X, T = _log_pairs()
    theta, l0, l1 = binding.cnn_train(ocnn.init_params(0), X, T, np.ones_like(T), steps=600, batch=8, lr=2e-3, seed=1)
    assert l1 < 0.1 * l0
    r1, mp1, mc1, d1 = _cnn_vs_plain(theta, 1)
    assert mp1 == 0 and mc1 == 0
    assert r1 < 1.0
    r2, mp2, mc2, d2 = _cnn_vs_plain(theta, 2)
    assert mp2 == 0 and mc2 == 0
    assert d2 <= 1e-4
