"""Parity of the CUDA demigration (the transpose of Eq. 1, Sec. 3 read from the data side)
with the FP64 oracle's transpose, element by element on seeded inputs, and the adjoint
dot-product identity between the two CUDA operators."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, cfg2_reduced, gpu_demigrate, gpu_migrate, rel_l2
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu

CASES = [
    # dim, ntr, nx, ny, nz, nt, vel, weight, aperture, n_bins
    (2, 60, 45, 1, 37, 200, "const", "one", 0.0, 3),
    (2, 80, 70, 1, 50, 300, "linear", "one", 0.0, 4),
    (2, 50, 33, 1, 65, 257, "linear", "obliq", 150.0, 2),
    (3, 90, 19, 21, 23, 240, "const", "obliq", 120.0, 3),
    (3, 300, 17, 18, 40, 320, "linear", "obliq", 140.0, 5),
    (3, 70, 33, 5, 17, 181, "linear", "one", 0.0, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{c[6]}-{c[7]}-A{int(c[8])}" for c in CASES])
@pytest.mark.parametrize("fast_math", [True, False])
def test_demigrate_random_surveys(case, fast_math):
    dim, ntr, nx, ny, nz, nt, vel, weight, ap, nb = case
    rng = np.random.default_rng(200 + ntr)
    s = sv.survey_random(rng, dim, ntr, nx, ny, nz, nt, vel=vel, weight=weight, aperture=ap,
                         n_bins=nb, h=12.5, v0=1700.0, k=0.6 if vel == "linear" else 0.0,
                         t0=0.008)
    m = sv.random_image(s, 5)
    got, _ = gpu_demigrate(s, m, fast_math=fast_math)
    want = oracle.demigrate(s, m)
    assert np.count_nonzero(want) > 0
    assert rel_l2(got, want) < FP32_REL_L2


def test_demigrate_3d_vz_reduced():
    s, d = cfg2_reduced()
    m = oracle.migrate(s, d)                 # a paper-shaped image (migrated reflections)
    got, _ = gpu_demigrate(s, m)
    assert rel_l2(got, oracle.demigrate(s, m.astype(np.float32))) < FP32_REL_L2


def test_adjoint_identity_between_cuda_operators():
    rng = np.random.default_rng(21)
    s = sv.survey_random(rng, 3, 400, 24, 20, 48, 400, vel="linear", weight="obliq",
                         aperture=160.0, n_bins=4, h=12.5, v0=1600.0, k=0.5)
    d = sv.random_traces(s, 1, smooth=3)
    m = sv.random_image(s, 2)
    Ld, p = gpu_migrate(s, d)
    Ltm, _ = gpu_demigrate(s, m, plan=p)
    lhs = float(np.vdot(Ld, m.astype(np.float64)))
    rhs = float(np.vdot(d.astype(np.float64), Ltm))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


def test_demigrate_deterministic_and_edges():
    rng = np.random.default_rng(22)
    s = sv.survey_random(rng, 2, 40, 31, 1, 29, 131, vel="linear", n_bins=2, h=10.0, k=0.5)
    m = sv.random_image(s, 3)
    a, p = gpu_demigrate(s, m)
    b, _ = gpu_demigrate(s, m, plan=p)
    assert np.array_equal(a, b)
    assert rel_l2(a, oracle.demigrate(s, m)) < FP32_REL_L2
    # offsets beyond the last bin: zero traces
    far = s.replace(bin_width=0.01)
    z, _ = gpu_demigrate(far, m)
    assert not np.any(z)
