"""True-amplitude weight (constant velocity) on the GPU against the FP64 oracle: migration of random
2D and 3D surveys element by element (apertures, taper, fast and exact square roots, sample pairs
on and off, 16-bit traces), demigration and the dot-product identity between the two CUDA
operators, a horizontal reflector whose image keeps its peak across offsets, and the refusals."""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, MIXED_REL_L2, gpu_demigrate, gpu_migrate, quantize, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu

CASES = [
    # dim, ntr, nx, ny, nz, nt, aperture, taper
    (3, 90, 19, 21, 35, 260, 0.0, 0.0),
    (3, 120, 33, 17, 20, 300, 150.0, 0.25),
    (2, 80, 70, 1, 53, 300, 0.0, 0.0),
    (2, 70, 45, 1, 40, 257, 120.0, 0.4),
]


def ta_survey(case, seed):
    dim, ntr, nx, ny, nz, nt, ap, taper = case
    rng = np.random.default_rng(seed)
    s = sv.survey_random(rng, dim, ntr, nx, ny, nz, nt, weight="ta", aperture=ap, n_bins=3, h=12.5, v0=1900.0)
    return s.replace(taper=taper)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-A{int(c[6])}-t{c[7]}" for c in CASES])
@pytest.mark.parametrize("fast_math", [True, False])
@pytest.mark.parametrize("pairs", [1, 0])
def test_migrate_matches_oracle(case, fast_math, pairs):
    s = ta_survey(case, 300 + case[1])
    d = sv.random_traces(s, 7, smooth=5)
    p = kh.Plan(s, fast_math=fast_math)
    p.set_option(kh.KH_OPT_SAMPLE_PAIRS, pairs)
    got, _ = gpu_migrate(s, d, plan=p)
    want = oracle.migrate(s, d)
    assert np.count_nonzero(want) > 0
    assert rel_l2(got, want) < FP32_REL_L2


def test_half_precision_traces():
    s = ta_survey(CASES[1], 41)
    d = sv.random_traces(s, 3, smooth=5)
    got, _ = gpu_migrate(s, d, trace_dtype=torch.float16)
    assert rel_l2(got, oracle.migrate(s, quantize(d, torch.float16))) < FP32_REL_L2
    assert rel_l2(got, oracle.migrate(s, d)) < MIXED_REL_L2


@pytest.mark.parametrize("case", CASES[1:3], ids=["3d", "2d"])
def test_demigrate_and_dot_product(case):
    s = ta_survey(case, 500 + case[1])
    d = sv.random_traces(s, 11, smooth=3)
    # element-wise parity on a migrated (coherent) image: a white-noise image makes every trace
    # sample a sum of terms of random sign whose FP32 rounding alone is near the bar in 2D (1.2e-5
    # for W = 1 as well on this survey)
    mc = oracle.migrate(s, d).astype(np.float32)
    got, p = gpu_demigrate(s, mc)
    assert rel_l2(got, oracle.demigrate(s, mc)) < FP32_REL_L2
    m = sv.random_image(s, 2)
    Ltm, _ = gpu_demigrate(s, m, plan=p)
    Ld, _ = gpu_migrate(s, d, plan=p)
    lhs = float(np.vdot(Ld, m.astype(np.float64)))
    rhs = float(np.vdot(d.astype(np.float64), Ltm))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))


def test_flat_reflector_keeps_its_peak():
    # 3D common-offset grids over a horizontal reflector at 500 m; data = R / (4 pi L) x the time
    # derivative of a 25 Hz Ricker at the specular time (the oracle's pin, on the GPU)
    v, zr, half, spacing = 2000.0, 500.0, 400.0, 10.0
    offsets = [100.0, 300.0, 500.0, 700.0]
    g = np.arange(-half, half + 1e-9, spacing)
    MX, MY = np.meshgrid(g, g, indexing="ij")
    mx, my = MX.ravel(), MY.ravel()
    sx = np.concatenate([mx - o / 2 for o in offsets]).astype(np.float32)
    rx = np.concatenate([mx + o / 2 for o in offsets]).astype(np.float32)
    sy = np.concatenate([my for _ in offsets]).astype(np.float32)
    dt, nt = 0.0005, 1600   # 0.8 s: past the largest specular time (0.61 s at 700 m)
    L = np.hypot(sx.astype(np.float64) - rx, 2 * zr)
    u = np.arange(nt)[None, :] * dt - (L / v)[:, None]
    ricker = (1 - 2 * (math.pi * 25 * u) ** 2) * np.exp(-(math.pi * 25 * u) ** 2)
    d = ((1.0 / (4 * math.pi * L))[:, None] * np.gradient(ricker, dt, axis=1)).astype(np.float32)
    s = sv.Survey(dim=3, nx=1, ny=1, nz=61, ox=0.0, oy=0.0, oz=zr - 30.0, dx=1.0, dy=1.0, dz=1.0, n_bins=4,
                  bin_width=200.0, vel="const", v0=v, k=0.0, weight="ta", r0=1000.0, aperture=half, nt=nt,
                  t0=0.0, dt=dt, sx=sx, sy=sy, rx=rx, ry=sy.copy(), taper=0.5)
    got, _ = gpu_migrate(s, d)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2
    peaks = np.abs(got).max(axis=(1, 2, 3))
    assert np.max(np.abs(peaks / peaks[0] - 1.0)) < 0.005


def test_refusals():
    rng = np.random.default_rng(3)
    s = sv.survey_random(rng, 3, 20, 8, 8, 16, 64, weight="ta")
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Plan(s.replace(vel="linear", k=0.5))
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    p = kh.Plan(s)
    hdr = kh.Headers.of(s)
    with pytest.raises(kh.KirchhoffError) as ei:
        p.velocity_grad(hdr, torch.zeros(p.image_shape, device="cuda"), torch.zeros((s.ntr, s.nt), device="cuda"))
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Batch([(p, hdr, torch.zeros((s.ntr, s.nt), device="cuda"), torch.zeros(p.image_shape, device="cuda"))])
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
