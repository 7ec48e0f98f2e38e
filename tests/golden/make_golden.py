"""Writes the oracle regression fixtures of this folder (``oracle_runs.json``).

The paper prints no solution values: its only tables are device-busy fractions
per machine (Sec. 5), so there is no worked example to store.  These fixtures
therefore pin the FP64 oracle to itself over time.  Each case is a small seeded
run of ``oracle/`` alone (no CUDA path).  ``tests/test_oracle_golden.py``
reruns the cases and compares, so any change to the oracle's arithmetic shows
up as a diff of this file, which the change then regenerates and justifies.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import platform
import sys

import numpy as np

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle                                        # noqa: E402
from paper_1901_06798_gb300 import workloads as W    # noqa: E402

OUT = os.path.join(os.path.dirname(__file__), "oracle_runs.json")


def _cases():
    """name -> (workload, steps, what the case exercises)."""
    hump = W.hump200()
    amr = W.amr3(L=240e3, dx1=4000.0, steps=12)
    shelf = W.shelf(n=96, dx=4000.0, steps=40)
    return {
        "hump200_split": (hump, 50, "Godunov-split update, all wet (Sec. 2.2)"),
        "hump200_unsplit": (dict(hump, cfg=dict(hump["cfg"], transverse=1)), 50,
                            "unsplit update with transverse corrections"),
        "shelf96_friction": (dict(shelf, cfg=dict(shelf["cfg"], manning_n=0.025)), 40,
                             "shelf with beach and dry land, uplift, Manning friction n = 0.025 (Sec. 2.1)"),
        "amr3_shelf240km": (amr, 12, "3-level AMR: flagging, clustering, ghost fill, averaging (Sec. 3.1)"),
        "hump200_lonlat": (W.lonlat(hump, lon0=140.0, lat0=35.0), 40,
                           "latitude-longitude capacity form"),
    }


def run_case(w, steps):
    o = W.load(oracle.Oracle(w["cfg"]), w)
    o.step(steps)
    st = o.stats()
    t, e = o.read_gauges()
    return {
        "steps": steps,
        "dt": st["dt"], "t": st["t"], "mass": st["mass"],
        "cell_updates": st["cell_updates"], "patches": st["patches"],
        "gauge_t": [float(v) for v in np.asarray(t).ravel()],
        "gauge_eta": [[float(v) for v in row] for row in np.asarray(e).reshape(len(t), -1)],
    }


def main():
    out = {"_machine": platform.machine()}
    for name, (w, steps, what) in _cases().items():
        out[name] = dict(run_case(w, steps), what=what)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
