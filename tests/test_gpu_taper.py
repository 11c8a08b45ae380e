"""The aperture taper on the GPU (the weight falls as a raised cosine over the outer part of the
aperture): migration, demigration and the velocity gradient against the FP64 oracle on random
surveys with every velocity kind that has them, the dot-product identity of the tapered pair,
and the hand values of the taper on one column."""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, GRAD_REL, gpu_demigrate, gpu_migrate, gpu_vgrad, rel_l2
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu

CASES = [
    # dim, vel, weight, aperture, taper
    (3, "linear", "obliq", 140.0, 0.3),
    (3, "const", "one", 120.0, 0.5),
    (2, "linear", "one", 150.0, 0.25),
    (3, "pstm", "obliq", 130.0, 0.4),
]


def _survey(case, seed):
    dim, vel, weight, ap, tp = case
    rng = np.random.default_rng(seed)
    s = sv.survey_random(rng, dim, 110, 30, 26 if dim == 3 else 1, 40, 300, vel=vel, weight=weight,
                         aperture=ap, n_bins=3, h=12.5, v0=1700.0, k=0.0 if vel == "const" else 0.6)
    s = s.replace(taper=tp)
    return s.replace(dz=0.01) if vel == "pstm" else s


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{c[1]}-{c[2]}-f{c[4]}" for c in CASES])
def test_tapered_migration(case):
    s = _survey(case, 300)
    d = sv.random_traces(s, 3, smooth=5)
    got, _ = gpu_migrate(s, d)
    want = oracle.migrate(s, d)
    assert rel_l2(want, oracle.migrate(s.replace(taper=0.0), d)) > 1e-3   # the taper matters here
    assert rel_l2(got, want) < FP32_REL_L2


@pytest.mark.parametrize("case", CASES[:3], ids=[f"{c[0]}d-{c[1]}-{c[2]}" for c in CASES[:3]])
def test_tapered_adjoint_and_gradient(case):
    s = _survey(case, 301)
    d = sv.random_traces(s, 4, smooth=9)
    m = sv.random_image(s, 5)
    got, _ = gpu_demigrate(s, m)
    assert rel_l2(got, oracle.demigrate(s, m)) < FP32_REL_L2
    img, _ = gpu_migrate(s, d)
    assert abs(np.vdot(img, m) - np.vdot(d, got)) <= 1e-5 * abs(np.vdot(img, m))
    if s.k != 0.0:
        g, _ = gpu_vgrad(s, m, d)
        want, ab = oracle.vgrad(s, m, d, return_abs=True)
        assert abs(g[0] - want[0]) <= GRAD_REL * ab[0] and abs(g[1] - want[1]) <= GRAD_REL * ab[1]


def test_taper_hand_values_on_one_column():
    for dist, want in ((100.0, 1.0), (187.5, 0.5 * (1 + math.cos(math.pi / 4))), (225.0, 0.5)):
        s = sv.Survey(dim=2, nx=1, ny=1, nz=1, ox=0.0, oy=0.0, oz=0.0, dx=10.0, dy=10.0, dz=10.0,
                      n_bins=1, bin_width=1e4, vel="const", v0=2500.0, k=0.0, weight="one", r0=1e3,
                      aperture=300.0, nt=400, t0=0.0, dt=0.004, sx=np.array([dist - 50.0], np.float32),
                      sy=np.zeros(1, np.float32), rx=np.array([dist + 50.0], np.float32),
                      ry=np.zeros(1, np.float32), taper=0.5)
        got, _ = gpu_migrate(s, np.ones((1, s.nt), np.float32))
        assert abs(got[0, 0, 0, 0] - want) < 1e-6, (dist, got[0, 0, 0, 0], want)
