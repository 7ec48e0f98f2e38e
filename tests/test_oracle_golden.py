"""The FP64 oracle against its stored regression fixtures
(``tests/golden/oracle_runs.json``, written by ``tests/golden/make_golden.py``
from ``oracle/`` alone).

The paper prints no solution values to pin against (its tables are device-busy
fractions), so these fixtures guard the oracle against unnoticed drift: the five
small runs (split and unsplit updates, friction over dry land, 3-level AMR,
latitude-longitude grid) must reproduce their stored steps, patch counts, mass
and gauge records.  On the machine type that wrote the fixtures the match is
bit for bit; elsewhere the last bits of the C library's exp, pow and sin may
differ, so the bar there is 1e-12 relative.
"""
import importlib.util
import json
import os
import platform

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


STORED = json.load(open(os.path.join(HERE, "oracle_runs.json")))
CASES = sorted(k for k in STORED if not k.startswith("_"))


@pytest.mark.parametrize("name", CASES)
def test_oracle_reproduces_stored_run(name):
    m = _maker()
    w, steps, _ = m._cases()[name]
    got = m.run_case(w, steps)
    ref = STORED[name]
    assert got["steps"] == ref["steps"]
    assert got["patches"] == ref["patches"]
    assert got["cell_updates"] == ref["cell_updates"]
    exact = platform.machine() == STORED["_machine"]
    for key in ("dt", "t", "mass", "gauge_t", "gauge_eta"):
        a, b = np.asarray(got[key], dtype=float), np.asarray(ref[key], dtype=float)
        assert a.shape == b.shape, key
        if exact:
            assert np.array_equal(a, b), key
        else:
            scale = max(np.abs(b).max(), 1e-300)
            assert np.abs(a - b).max() <= 1e-12 * scale, key


def test_fixtures_cover_every_case():
    assert CASES == sorted(_maker()._cases())
