"""Pins of two properties Sec. 2.2 states for the method, held against the
mathematics rather than against the oracle itself.

1. The Riemann solver keeps depths non-negative.  The solver's waves define a
   fan of constant states: left state, the state after the 1-wave, the states
   on either side of the stationary bed-step wave at x = 0, the state before
   the 3-wave, right state.  Each state is recovered from the solver's output
   alone (f-wave / speed = wave; the stationary wave carries the rest of the
   depth jump) and must have h >= 0, on bed steps, dry fronts, overtopping and
   supersonic flow.  Built on that solver, the first-order update of
   Eq. (wave_propagation_form) is a convex combination of those states when no
   wave crosses more than half a cell, so it must keep h >= 0 too.

2. The CFL condition nu <= 1 must hold.  A level-1 step that breaks it is
   discarded and taken again with dt = cfl_desired / (s / dx) from the speeds
   it saw.  At a dam break onto a dry bed the first step's dt comes from the
   cell speeds sqrt(g h), but the front runs at 2 sqrt(g h) (Ritter), so the
   first step must be retaken, and the kept step's dt is the closed form
   cfl_desired dx / (2 sqrt(g h)).
"""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import workloads as W

G = 9.81
DRYTOL = 1e-3


def fan_depths(hL, hnL, BL, hR, hnR, BR):
    """Depths of the constant states of the solver's fan, from its output.

    With a wall the dry side is the mirror of the wet one (same bed).  W^p =
    Z^p / s^p (mass component); the stationary wave carries
    delta = (hR - hL) - W1 - W3.  Returns None for two dry cells (no fan)."""
    Z, s, wl, wr = oracle.riemann(hL, hnL, 0.0, BL, hR, hnR, 0.0, BR)
    if hL < DRYTOL and hR < DRYTOL:
        return None
    if wr:
        hR, hnR, BR = hL, -hnL, BL
    if wl:
        hL, hnL, BL = hR, -hnR, BR
    s1, s3 = s[0], s[2]
    assert s1 < s3
    if s1 == 0.0 or s3 == 0.0:
        return None   # the wave cannot be recovered from its f-wave (measure zero)
    W1, W3 = Z[0][0] / s1, Z[2][0] / s3
    delta = (hR - hL) - W1 - W3
    if s1 < 0.0 < s3:
        states = [hL + W1, hR - W3]   # either side of the bed step
    elif s1 > 0.0:
        states = [hL + delta, hL + delta + W1]
    else:
        states = [hL + W1, hR - delta]
    return [hL, hR] + states


def _tol(*h):
    return 1e-12 * max(1.0, *[abs(v) for v in h])


def test_fan_depths_non_negative_on_bed_steps_dry_fronts_and_overtopping():
    cases = {
        # deep water running away from a shallow shelf: with a continuous surface the
        # shelf side of the bed step would go negative, so the bound must hold it at 0
        "draining shelf": (1.0, -1.0, -1.0, 0.01, 0.0, -0.01),
        # supersonic flow (Froude 3.6) at a step 0.8 m above its bed, higher than its surface
        "supersonic up a step": (0.5, 0.5 * 8.0, -0.5, 0.5, 0.5 * 8.0, 0.3),
        # the same flow mirrored: supersonic to the left, all waves left-going
        "supersonic up a step, mirrored": (0.5, -0.5 * 8.0, 0.3, 0.5, -0.5 * 8.0, -0.5),
        # still water next to a dry cell 1 m lower: the dry bed floods down the step
        "dry front down a step": (1.0, 0.0, -1.0, 0.0, 0.0, -2.0),
        # 1 m of water at 3 m/s running at a dry step 2 m above its bed (it overtops)
        "overtopping a dry step": (1.0, 3.0, -5.0, 0.0, 0.0, -3.0),
        "overtopping, mirrored": (0.0, 0.0, -3.0, 1.0, -3.0, -5.0),
    }
    at_bound = 0
    for name, (hL, hnL, BL, hR, hnR, BR) in cases.items():
        d = fan_depths(hL, hnL, BL, hR, hnR, BR)
        assert d is not None
        assert min(d) >= -_tol(hL, hR), (name, d)
        at_bound += abs(min(d)) <= _tol(hL, hR)
    # the draining shelf, both supersonic cases and the dry front need the bound:
    # one state of each fan sits exactly at zero depth
    assert at_bound >= 4
    # the bound moves the bed-step jump only as far as needed: the state that
    # would go negative is the one held at zero, on whichever side it lies
    for hL, hnL, BL, hR, hnR, BR, zero_side in ((1.0, -1.0, -1.0, 0.01, 0.0, -0.01, 1),
                                                (0.01, 0.0, -0.01, 1.0, 1.0, -1.0, 0)):
        d = fan_depths(hL, hnL, BL, hR, hnR, BR)
        assert abs(d[2 + zero_side]) <= _tol(hL, hR) and d[3 - zero_side] > 1e-3, d

    rng = np.random.default_rng(2008)
    n_bounded = 0
    for _ in range(20000):
        hL = rng.uniform(0, 0.002) if rng.random() < 0.25 else rng.uniform(0, 5)
        hR = rng.uniform(0, 0.002) if rng.random() < 0.25 else rng.uniform(0, 5)
        BL = rng.uniform(-5, 1)
        BR = BL + (rng.uniform(-4, 4) if rng.random() < 0.8 else 0.0)
        hnL = hL * rng.uniform(-10, 10) if hL >= DRYTOL else 0.0
        hnR = hR * rng.uniform(-10, 10) if hR >= DRYTOL else 0.0
        d = fan_depths(hL, hnL, BL, hR, hnR, BR)
        if d is None:
            continue
        assert min(d) >= -_tol(hL, hR), ((hL, hnL, BL, hR, hnR, BR), d)
        n_bounded += abs(min(d[2:])) <= _tol(hL, hR) and min(hL, hR) >= DRYTOL
    assert n_bounded > 100   # the random problems do reach the bound


def _first_order_step(h, hn, B, nu):
    """One first-order step of Eq. (wave_propagation_form) with the oracle's
    solver, dt = nu dx / max |s|: h_i - dt/dx (A+dQ_{i-1/2} + A-dQ_{i+1/2})
    (mass component; a wave of speed 0 splits half to each side; a wall edge
    sends nothing into its dry side)."""
    n = len(h)
    am, ap, smax = np.zeros(n - 1), np.zeros(n - 1), 0.0
    for e in range(n - 1):
        Z, s, wl, wr = oracle.riemann(h[e], hn[e], 0.0, B[e], h[e + 1], hn[e + 1], 0.0, B[e + 1])
        left = [1.0 if sp < 0 else (0.5 if sp == 0 else 0.0) for sp in s]
        am[e] = sum(left[p] * Z[p][0] for p in range(3))
        ap[e] = sum((1.0 - left[p]) * Z[p][0] for p in range(3))
        if wr:
            ap[e] = 0.0
        if wl:
            am[e] = 0.0
        smax = max(smax, -s[0], s[2])
    if smax == 0.0:
        return h[1:-1].copy()
    dtdx = nu / smax
    return h[1:-1] - dtdx * (ap[:-1] + am[1:])


def test_first_order_update_keeps_depth_non_negative():
    """Random channels of 8 cells over stepped beds with dry cells, at
    Courant number 1/2: no updated depth is negative (up to rounding)."""
    rng = np.random.default_rng(1901)
    worst = 0.0
    for _ in range(3000):
        n = 8
        h = np.where(rng.random(n) < 0.3, rng.uniform(0, 0.002, n), rng.uniform(0, 3, n))
        B = np.cumsum(rng.choice([0, 1], n) * rng.uniform(-3, 3, n)) - 2.0
        hn = np.where(h >= DRYTOL, h * rng.uniform(-4, 4, n), 0.0)
        hnew = _first_order_step(h, hn, B, 0.5)
        worst = min(worst, float(hnew.min()))
    assert worst >= -1e-12, worst


# --------------------------------------------------------------------------
# CFL retake

def _ritter(n=200, cfl_retake=1):
    w = W.dam_break_1d(n, 1.0, 0.0)
    cfg = dict(w["cfg"], cfl_retake=cfl_retake)
    return W.load(oracle.Oracle(cfg), dict(w, cfg=cfg)), cfg


def test_dam_break_onto_dry_bed_retakes_its_first_step():
    o, cfg = _ritter()
    t = o.step(1)[0]
    st = o.stats()
    c = np.sqrt(G * 1.0)
    assert st["cfl_retakes"] == 1 and st["cfl_violations"] == 0
    assert abs(t - 0.9 * cfg["dx"] / (2.0 * c)) <= 1e-14 * t
    # the next steps keep nu <= cfl_max; a retake may recur as the front speeds up
    for _ in range(30):
        o.step(1)
    assert o.stats()["cfl_violations"] == 0
    # the retaken step is the step taken from the same state with the smaller dt
    o3, _ = _ritter()
    w = W.dam_break_1d(200, 1.0, 0.0)
    cfg3 = dict(w["cfg"], dt_max=t)   # the retaken step's dt, the closed form above to rounding
    o4 = W.load(oracle.Oracle(cfg3), dict(w, cfg=cfg3))
    assert np.array_equal(o3.step(1), o4.step(1))
    assert o4.stats()["cfl_retakes"] == 0
    for f in ("h", "hu", "hv"):
        assert np.array_equal(o3.level_array(0, 1, f), o4.level_array(0, 1, f)), f
    # without retakes the same first step is kept and counted
    o2, _ = _ritter(cfl_retake=0)
    t2 = o2.step(1)[0]
    assert o2.stats()["cfl_violations"] == 1 and o2.stats()["cfl_retakes"] == 0
    assert abs(t2 - 0.9 * cfg["dx"] / c) <= 1e-14 * t2


def test_retake_keeps_courant_number_below_the_limit_on_a_beach():
    """A wave running up a dry beach: thin films make the wave speed jump from
    one step to the next, past what cfl_desired leaves room for.  Retakes
    happen during the run-up (not only at t = 0), and every kept level-1 step
    has nu <= cfl_max; without retakes the same run keeps violating steps."""
    w = W.beach_runup()
    o = W.load(oracle.Oracle(w["cfg"]), w)
    o.step(1)
    assert o.stats()["cfl_retakes"] == 0
    o.step(39)
    st = o.stats()
    assert st["cfl_violations"] == 0
    assert st["cfl_retakes"] >= 2
    w0 = W.beach_runup(cfl_retake=0)
    o0 = W.load(oracle.Oracle(w0["cfg"]), w0)
    o0.step(40)
    assert o0.stats()["cfl_violations"] >= 1
