"""Write tests/golden/tiny_city_oracle.json: the oracle's results on the tiny
city (8x8 box buildings, 32x32 microphones at 1.5 m) -- one source with
level-4 beams and reflection order 4, and two sources with level-6 beams and
order 5 -- the small-city problem of Section 4 at sizes the oracle traces in
seconds.  Per case: the segment count, every microphone's path count, and the
band levels of every microphone reached.

The file is a regression record of the oracle, not a pin: the pins are the
closed forms and brute-force enumerations of test_oracle_pins.py.  It makes
any change of the oracle's arithmetic visible.  A change that is meant
regenerates the file with this script (python tests/golden/make_oracle_golden.py),
and its commit message names the passage of the paper that justifies it.
Only the oracle and the seeded input generator are called here.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1912_03998_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_city_oracle.json")
# (seed, beam level L, maximum reflection order K, sources)
CASES = [(1, 4, 4, 1), (2, 6, 5, 2)]


def workload(seed, level, max_order, n_sources):
    return synth.tiny_city(seed=seed, level=level, max_order=max_order, n_sources=n_sources)


def compute_case(seed, level, max_order, n_sources):
    w = workload(seed, level, max_order, n_sources)
    r = oracle.trace_workload(w)
    L = oracle.levels(r["I"])
    reached = np.flatnonzero(r["cnt"] > 0)
    return {
        "workload": {"name": "tiny_city", "seed": seed, "level": level, "max_order": max_order,
                     "n_sources": n_sources, "n_mics": int(len(w.mics)), "n_tris": int(len(w.scene.tris))},
        "segments": int(r["stats"]["segments"]),
        "count": [int(c) for c in r["cnt"]],
        "reached": [int(i) for i in reached],
        "level_db": [[float(f"{x:.10g}") for x in L[i]] for i in reached],
    }


def compute():
    return {"cases": [compute_case(*c) for c in CASES]}


if __name__ == "__main__":
    d = compute()
    with open(OUT, "w") as f:
        json.dump(d, f, separators=(",", ":"))
        f.write("\n")
    for c in d["cases"]:
        print(f"{c['workload']}: {c['segments']} segments, {len(c['reached'])} microphones reached")
