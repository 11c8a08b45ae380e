"""Tile autotuner host logic (no GPU): bucket keys and the JSON cache."""
import json

import numpy as np

import torch

from paper_1204_1225_gb300.autotune import CANDIDATES, TileTuner, bucket_key
from paper_1204_1225_gb300.survey import survey_3d_gradient, survey_batch_3d


class _FakePlan:
    def __init__(self, s):
        self.survey = s
        self.trace_dtype = torch.float32
        self.tile = None

    def set_tile(self, t):
        self.tile = t


def test_bucket_key_groups_and_separates():
    a = survey_3d_gradient(100, 128).replace(nt=1500)
    assert bucket_key(a) == bucket_key(a.replace(nt=1100))          # same nt bucket (2048)
    assert bucket_key(a) != bucket_key(a.replace(nt=900))           # 1024 bucket
    assert bucket_key(a) != bucket_key(a, torch.float16)
    assert bucket_key(a) != bucket_key(survey_3d_gradient(100, 192))
    assert bucket_key(a) != bucket_key(a.replace(k=0.0))


def test_every_candidate_has_256_threads():
    for dim, cs in CANDIDATES.items():
        for cx, cy, cz in cs:
            assert cx * cy * cz == 256 and cz <= 16 and (dim == 3 or cy == 1)


def test_cache_hit_sets_tile_without_timing(tmp_path):
    s = survey_3d_gradient(100, 96)
    path = tmp_path / "t.json"
    path.write_text(json.dumps({bucket_key(s): {"tile": [8, 8, 4], "ms": {}}}))
    tuner = TileTuner(path=str(path))
    plan = _FakePlan(s)
    assert tuner.choose(plan, None, None) == (8, 8, 4)
    assert plan.tile == (8, 8, 4) and tuner.timed == 0


def test_batch_generator_is_seeded_and_in_range():
    a, b = survey_batch_3d(8), survey_batch_3d(8)
    assert [(j.nx, j.ntr, j.nt) for j in a] == [(j.nx, j.ntr, j.nt) for j in b]
    for j in survey_batch_3d(64):
        assert 64 <= j.nx <= 192 and 1000 <= j.ntr <= 50_000 and 750 <= j.nt <= 2000
        assert j.nx == j.ny == j.nz and j.dx == 10.0 and j.vel == "const" and j.aperture == 0.0
        w = j.nx * j.dx
        assert 0 <= j.sx.min() and j.sx.max() < w and 0 <= j.ry.min() and j.ry.max() < w
        off = np.hypot(j.sx.astype(np.float64) - j.rx, j.sy.astype(np.float64) - j.ry)
        assert off.max() < j.n_bins * j.bin_width
