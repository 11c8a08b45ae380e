"""Writes oracle_2d_const_samples.json: FP64 oracle values of Eq. 1 (Sec. 3) at 64 seeded
image samples of the seeded 2D constant-velocity survey (16 shots x 64 receivers, 3 point
diffractors, 25 Hz Ricker, noise sigma 0.1).  Calls only the oracle and the seeded input
generators; a regression fixture for the oracle, not a pin.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1204_1225_gb300 import survey as sv  # noqa: E402


def main():
    s = sv.survey_2d_const()
    sc = sv.point_scatterers_2d(np.random.default_rng(sv.BASE_SEED))
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0, noise_sigma=0.1, seed=sv.BASE_SEED).numpy()
    idx = sv.sample_points(s, 64, seed=sv.BASE_SEED + 1)
    val = oracle.migrate_points(s, d, idx)
    out = {
        "cite": "Eq. 1 (Sec. 3): offset-binned Kirchhoff sum; FP64 oracle",
        "survey": s.name, "seed": sv.BASE_SEED, "freq_hz": 25.0, "noise_sigma": 0.1,
        "flat_index": [int(i) for i in idx], "value": [float(v) for v in val],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                           "oracle_2d_const_samples.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
