"""The oracle still produces the stored FP64 values (written by tests/golden/make_golden.py)."""
import json
import os

import numpy as np

import oracle
from paper_1204_1225_gb300 import survey as sv

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_samples():
    g = json.load(open(os.path.join(HERE, "golden", "oracle_2d_const_samples.json")))
    s = sv.survey_2d_const()
    sc = sv.point_scatterers_2d(np.random.default_rng(g["seed"]))
    d = sv.synthesize(s, sc, oracle.arrival_times, g["freq_hz"], noise_sigma=g["noise_sigma"],
                      seed=g["seed"]).numpy()
    val = oracle.migrate_points(s, d, np.array(g["flat_index"], dtype=np.int64))
    assert np.allclose(val, g["value"], rtol=1e-12, atol=1e-9)
