"""The oracle reproduces its stored results on the tiny city
(tests/golden/tiny_city_oracle.json, written by
tests/golden/make_oracle_golden.py from the oracle alone).  A regression
record, not a pin: it flags any change of the oracle's arithmetic, which then
regenerates the file with the script and names the passage of the paper that
justifies it."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "tiny_city_oracle.json")


def _script():
    spec = importlib.util.spec_from_file_location("make_oracle_golden",
                                                  os.path.join(HERE, "golden", "make_oracle_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


with open(GOLDEN) as f:
    STORED = json.load(f)["cases"]


@pytest.mark.parametrize("case", STORED, ids=lambda c: f"L{c['workload']['level']}K{c['workload']['max_order']}")
def test_oracle_matches_stored_result(oracle_mod, case):
    m = _script()
    wl = case["workload"]
    got = m.compute_case(wl["seed"], wl["level"], wl["max_order"], wl["n_sources"])
    assert got["workload"] == wl
    assert got["segments"] == case["segments"]
    assert got["count"] == case["count"]
    assert got["reached"] == case["reached"]
    a, b = np.array(got["level_db"]), np.array(case["level_db"])
    assert a.shape == b.shape and np.abs(a - b).max(initial=0.0) < 1e-6


def test_stored_results_are_plausible():
    # levels of reached microphones are finite, a count is never negative, and
    # the reached list is exactly the microphones with a nonzero count
    for c in STORED:
        assert min(c["count"]) >= 0
        assert all(np.isfinite(c["level_db"]).ravel())
        assert [i for i, n in enumerate(c["count"]) if n > 0] == c["reached"]
