"""Prestack time migration (Sec. 4's PKTM) on the GPU against the FP64 oracle: random 2D and 3D
surveys with both weights and apertures, element by element; at k = 0 the time image equals the
constant-velocity depth image on the mapped axis z = v0 t0 / 2 (the library's own two paths);
a diffractor focuses at its (x, t0); the traveltime utility; refusals of the adjoint paths."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, gpu_migrate, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu

CASES = [
    # dim, ntr, nx, ny, nz, nt, weight, aperture, k
    (2, 70, 45, 1, 53, 300, "one", 0.0, 0.5),
    (2, 60, 33, 1, 40, 257, "obliq", 150.0, 0.8),
    (3, 90, 19, 21, 35, 240, "obliq", 120.0, 0.6),
    (3, 80, 17, 18, 20, 320, "one", 0.0, 0.0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{c[6]}-A{int(c[7])}-k{c[8]}" for c in CASES])
@pytest.mark.parametrize("fast_math", [True, False])
def test_random_surveys(case, fast_math):
    dim, ntr, nx, ny, nz, nt, weight, ap, k = case
    rng = np.random.default_rng(200 + ntr)
    s = sv.survey_random(rng, dim, ntr, nx, ny, nz, nt, vel="pstm", weight=weight, aperture=ap,
                         n_bins=3, h=12.5, v0=1700.0, k=k, t0=0.004).replace(oz=0.01, dz=0.012)
    d = sv.random_traces(s, 9, smooth=5)
    got, _ = gpu_migrate(s, d, fast_math=fast_math)
    want = oracle.migrate(s, d)
    assert np.count_nonzero(want) > 0
    assert rel_l2(got, want) < FP32_REL_L2


def test_constant_velocity_time_image_is_the_depth_image():
    rng = np.random.default_rng(7)
    s = sv.survey_random(rng, 3, 120, 24, 20, 48, 400, vel="pstm", weight="obliq", aperture=140.0,
                         n_bins=3, h=12.5, v0=2000.0, k=0.0).replace(oz=0.0, dz=0.0125)
    d = sv.random_traces(s, 3, smooth=5)
    depth = s.replace(vel="const", dz=s.v0 * s.dz / 2)
    t_img, _ = gpu_migrate(s, d)
    z_img, _ = gpu_migrate(depth, d)
    # the two FP32 paths evaluate the legs differently (time migration relative to the tile
    # centre); each agrees with the FP64 depth image of the oracle, and so with the other
    want = oracle.migrate(depth, d)
    assert rel_l2(t_img, want) < FP32_REL_L2 and rel_l2(z_img, want) < FP32_REL_L2
    assert rel_l2(t_img, z_img) < FP32_REL_L2


def test_diffractor_focuses_at_its_time():
    s = sv.survey_2d_const().replace(vel="pstm", v0=1800.0, k=0.4, oz=0.0, dz=0.008, nz=160)
    sc = np.array([[640.0, 0.0, 0.6, 1.0], [320.0, 0.0, 0.96, 1.0]])
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0).numpy()
    got, _ = gpu_migrate(s, d)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2
    stack = got.sum(axis=0)[0]
    for x, _, t0, _ in sc:
        ix, it = int(round(x / s.dx)), int(round(t0 / s.dz))
        assert stack[ix, it] == stack[ix - 2:ix + 3, it - 2:it + 3].max()


def test_traveltime_utility_and_refusals():
    rng = np.random.default_rng(8)
    s = sv.survey_random(rng, 3, 4, 8, 8, 8, 64, vel="pstm", v0=1500.0, k=0.55)
    p = kh.Plan(s)
    n = 3000
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda")
    px, py, lx, ly = (rng.uniform(-2000, 2000, n) for _ in range(4))
    t0 = rng.uniform(0.0, 3.0, n)
    T = p.traveltime(f(px), f(py), f(t0), f(lx), f(ly)).double().cpu().numpy()
    P = lambda a: np.asarray(a, np.float32).astype(np.float64)
    h = np.hypot(P(px) - P(lx), P(py) - P(ly))
    assert rel_l2(T, oracle.traveltime(s, h, P(t0))) < 1e-7
    hdr = kh.Headers.of(s)
    with pytest.raises(kh.KirchhoffError) as ei:
        p.demigrate(hdr, torch.zeros(p.image_shape, device="cuda"))
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Plan(s.replace(oz=-0.1))
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
