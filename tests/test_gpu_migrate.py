"""Parity of the CUDA migration (Eq. 1) with the FP64 oracle, element by element, on
seeded inputs: the 2D constant-velocity survey at full size, randomised 2D/3D surveys with
ragged tile tails, v(z) traveltimes, the obliquity-spreading weight and the aperture, and
the edge cases of the method (empty input, offsets beyond the last bin, two-sample traces,
unaligned rows, time-window edges)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, cfg1_inputs, gpu_migrate, rel_l2
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fast_math", [True, False])
def test_cfg1_full_image(fast_math):
    s, d = cfg1_inputs()
    got, _ = gpu_migrate(s, d, fast_math=fast_math)
    want = oracle.migrate(s, d)
    assert rel_l2(got, want) < FP32_REL_L2


def test_cfg1_deterministic():
    s, d = cfg1_inputs()
    a, p = gpu_migrate(s, d)
    b, _ = gpu_migrate(s, d, plan=p)
    assert np.array_equal(a, b)


CASES = [
    # dim, ntr, nx, ny, nz, nt, vel, weight, aperture, n_bins
    (2, 60, 45, 1, 37, 200, "const", "one", 0.0, 3),
    (2, 80, 70, 1, 50, 300, "linear", "one", 0.0, 4),
    (2, 50, 33, 1, 65, 257, "linear", "obliq", 150.0, 2),
    (3, 90, 19, 21, 23, 240, "const", "obliq", 120.0, 3),
    (3, 120, 17, 18, 40, 320, "linear", "obliq", 140.0, 5),
    (3, 70, 33, 5, 17, 181, "linear", "one", 0.0, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{c[6]}-{c[7]}-A{int(c[8])}" for c in CASES])
@pytest.mark.parametrize("fast_math", [True, False])
def test_random_surveys(case, fast_math):
    dim, ntr, nx, ny, nz, nt, vel, weight, ap, nb = case
    rng = np.random.default_rng(100 + ntr)
    s = sv.survey_random(rng, dim, ntr, nx, ny, nz, nt, vel=vel, weight=weight, aperture=ap,
                         n_bins=nb, h=12.5, v0=1700.0, k=0.6 if vel == "linear" else 0.0,
                         t0=0.008)
    d = sv.random_traces(s, 7, smooth=5)
    got, _ = gpu_migrate(s, d, fast_math=fast_math)
    want = oracle.migrate(s, d)
    assert np.count_nonzero(want) > 0
    assert rel_l2(got, want) < FP32_REL_L2


@pytest.mark.parametrize("tile", [(32, 1, 8), (64, 1, 4), (128, 1, 2)])
def test_tile_shapes_2d(tile):
    rng = np.random.default_rng(5)
    s = sv.survey_random(rng, 2, 64, 75, 1, 90, 300, vel="linear", n_bins=3, h=10.0, k=0.5)
    d = sv.random_traces(s, 3, smooth=5)
    got, _ = gpu_migrate(s, d, tile=tile)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2


@pytest.mark.parametrize("tile", [(16, 16, 1), (8, 8, 4), (32, 8, 1), (16, 8, 2)])
def test_tile_shapes_3d(tile):
    rng = np.random.default_rng(6)
    s = sv.survey_random(rng, 3, 60, 21, 19, 35, 300, vel="linear", weight="obliq", aperture=120.0,
                         n_bins=3, h=12.5, k=0.5)
    d = sv.random_traces(s, 4, smooth=5)
    got, _ = gpu_migrate(s, d, tile=tile)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2


def test_oversized_tile_is_refused_cleanly():
    from paper_1204_1225_gb300 import kirchhoff as kh
    rng = np.random.default_rng(6)
    s = sv.survey_random(rng, 3, 20, 8, 8, 256, 600, vel="linear", n_bins=2, h=25.0, k=0.8)
    d = sv.random_traces(s, 4)
    with pytest.raises(kh.KirchhoffError) as ei:
        gpu_migrate(s, d, tile=(4, 4, 16))
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    got, _ = gpu_migrate(s, d)          # the default tile adapts to the same survey
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2


def test_empty_and_out_of_range_inputs():
    rng = np.random.default_rng(8)
    s = sv.survey_random(rng, 3, 30, 10, 9, 20, 100, n_bins=2)
    d = sv.random_traces(s, 1)
    # no traces at all: a zero image
    e = s.subset(np.arange(0))
    got, _ = gpu_migrate(e, np.zeros((0, s.nt), np.float32))
    assert got.shape == s.image_shape and not np.any(got)
    # every offset beyond the last bin: nothing is imaged
    far = s.replace(bin_width=0.01)
    got, _ = gpu_migrate(far, d)
    assert not np.any(got) and not np.any(oracle.migrate(far, d))


def test_two_sample_traces_and_unaligned_rows():
    rng = np.random.default_rng(9)
    for nt in (2, 3, 5, 131):
        s = sv.survey_random(rng, 2, 25, 20, 1, 30, nt, n_bins=2, h=5.0, dt=0.002)
        d = sv.random_traces(s, nt)
        got, _ = gpu_migrate(s, d)
        want = oracle.migrate(s, d)
        if np.any(want):
            assert rel_l2(got, want) < FP32_REL_L2
        else:
            assert np.max(np.abs(got)) < 1e-6


def test_time_window_edges_exact():
    # zero-offset trace, v = 2000 m/s, dt = 4 ms: tau = z/4 exactly; D[i] = i + 1, nt = 101
    s = sv.Survey(dim=2, nx=1, ny=1, nz=110, ox=0.0, oy=0.0, oz=0.0, dx=4.0, dy=4.0, dz=4.0,
                  n_bins=1, bin_width=100.0, vel="const", v0=2000.0, k=0.0, weight="one", r0=1e3,
                  aperture=0.0, nt=101, t0=0.0, dt=0.004, sx=np.zeros(1, np.float32),
                  sy=np.zeros(1, np.float32), rx=np.zeros(1, np.float32), ry=np.zeros(1, np.float32))
    d = (1.0 + np.arange(101, dtype=np.float32))[None, :]
    got, _ = gpu_migrate(s, d)
    want = oracle.migrate(s, d)
    assert np.allclose(got, want, rtol=2e-6, atol=1e-4)
    assert got[0, 0, 0, 100] == pytest.approx(101.0, rel=1e-6)   # tau = nt - 1 is kept
    assert got[0, 0, 0, 101] == 0.0                              # tau = nt - 1 + 1 is not


def test_count_matches_oracle():
    from paper_1204_1225_gb300 import kirchhoff as kh
    rng = np.random.default_rng(10)
    s = sv.survey_random(rng, 3, 200, 40, 30, 7, 64, aperture=150.0, n_bins=4, h=12.5)
    p = kh.Plan(s)
    assert p.count(kh.Headers.of(s)) == oracle.count(s)


def test_traveltime_entry_matches_oracle():
    from paper_1204_1225_gb300 import kirchhoff as kh
    rng = np.random.default_rng(11)
    s = sv.survey_random(rng, 3, 4, 8, 8, 8, 64, vel="linear", k=0.55, v0=1500.0)
    p = kh.Plan(s)
    n = 5000
    px, py = rng.uniform(-2000, 2000, n), rng.uniform(-2000, 2000, n)
    pz = rng.uniform(0, 3000, n)
    lx, ly = rng.uniform(-2000, 2000, n), rng.uniform(-2000, 2000, n)
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda")
    T = p.traveltime(f(px), f(py), f(pz), f(lx), f(ly)).double().cpu().numpy()
    P = lambda a: np.asarray(a, np.float32).astype(np.float64)
    R = np.sqrt((P(px) - P(lx)) ** 2 + (P(py) - P(ly)) ** 2 + P(pz) ** 2)
    assert rel_l2(T, oracle.traveltime(s, R, P(pz))) < 1e-7


def test_wait_timeout_is_reported_and_context_survives():
    from paper_1204_1225_gb300 import kirchhoff as kh
    s, d = cfg1_inputs()
    s = s.replace(n_bins=1, bin_width=320.0)      # one bin of 1024 traces: many ring stages
    p = kh.Plan(s)
    hdr = kh.Headers.of(s)
    dt = torch.as_tensor(d, device="cuda")
    p.set_option(kh.KH_OPT_WAIT_POLLS, 1)
    p.migrate(hdr, dt)
    with pytest.raises(kh.KirchhoffError) as ei:
        p.sync()
    assert ei.value.status == kh.KH_ERR_TIMEOUT
    p.set_option(kh.KH_OPT_WAIT_POLLS, 0)
    img = p.migrate(hdr, dt)
    p.sync()
    assert rel_l2(img.double().cpu().numpy(), oracle.migrate(s, d)) < FP32_REL_L2


def test_aperture_hand_geometry_and_count():
    # the hand geometry of the oracle's aperture pin: trace j carries the constant 2^j, so the
    # image at every depth is the sum of the codes of the traces the aperture keeps (the
    # midpoint within A = 300 m of the column, <= inside, horizontal distance only)
    from paper_1204_1225_gb300 import kirchhoff as kh
    from test_oracle_pins import APERTURE_TRACES, aperture_survey
    s = aperture_survey()
    codes = 2.0 ** np.arange(len(APERTURE_TRACES))
    d = np.repeat(codes[:, None], s.nt, axis=1).astype(np.float32)
    want = sum(c for c, (_, kept) in zip(codes, APERTURE_TRACES) if kept)
    got, p = gpu_migrate(s, d)
    assert np.allclose(got[0, 0, 0], want, rtol=1e-6, atol=0), got[0, 0, 0]
    assert p.count(kh.Headers.of(s)) == sum(kept for _, kept in APERTURE_TRACES) * s.nz
    # a row of nine columns with one midpoint at x = 50 and A = 250: six columns (hand count)
    row = s.replace(dim=2, nx=9, ox=-400.0, dx=100.0, nz=3, aperture=250.0,
                    sx=np.zeros(1, np.float32), sy=np.zeros(1, np.float32),
                    rx=np.full(1, 100.0, np.float32), ry=np.zeros(1, np.float32))
    assert kh.Plan(row).count(kh.Headers.of(row)) == 6 * row.nz
