"""Gridded model v(x, z) on the GPU against the FP64 oracle: the eikonal solver's first-arrival
tables node by node (within the bound that the kernel's FP32 evaluation of the source-gradient
shift implies), migration with the per-location tables element by element over several models, node
spacings, weights, apertures and trace types, a diffractor under a low-velocity lens that focuses
with the tables and not with the background model, and the refusals and the missing-location
report."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, gpu_migrate, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu

MIXED_REL_L2 = 3e-3
# relative error of the kernel's FP32 shift h grad T0 = h s0 (dx, z) / r: the FP64 offset rounded to
# FP32 (2^-24), rsqrtf (2 ulp) and two products (2^-24 each)
EPS_SHIFT = 5e-7


def snapped_survey(seed, ntr, nx, nz, nt, h=10.0, weight="one", aperture=0.0, taper=0.0, snap=5.0):
    rng = np.random.default_rng(seed)
    s = sv.survey_random(rng, 2, ntr, nx, 1, nz, nt, weight=weight, aperture=aperture, n_bins=3, h=h,
                         v0=1800.0, k=0.5)
    f = lambda a: (np.round(a / snap) * snap).astype(np.float32)
    return s.replace(sx=f(s.sx), rx=f(s.rx), taper=taper)


def fp32_ulp(x):
    x = np.abs(np.asarray(x, np.float32))
    return np.spacing(x).astype(np.float64)


@pytest.mark.parametrize("m", [1, 2, 4])
@pytest.mark.parametrize("model", ["lens", "lateral"])
def test_tables_match_oracle(m, model):
    s = snapped_survey(31 + m, 40, 37, 41, 300, h=10.0)
    kw = dict(lens_dv=-500.0, lens_r=80.0) if model == "lens" else dict(lens_dv=0.0, lateral=0.4)
    s = sv.vxz_model(s, m, **kw)
    p = kh.Plan(s)
    T, r = p.grid_tables()
    T, r = T.double().cpu().numpy().transpose(0, 2, 1), r.cpu().numpy()   # stored [row][column]
    ref = oracle.grid_tables(s)
    assert np.all(np.abs(r - ref.rounds) <= 1)
    # tau and the node equation are FP64 as in the oracle; the kernel evaluates the shift
    # h grad T0 per update in FP32 (relative error <= EPS_SHIFT, so <= EPS_SHIFT h s0 per node),
    # and the update is 1-Lipschitz in each shifted neighbour, so the difference is at most that
    # per-node error times the longest upwind chain (nx + nz nodes), plus the FP32 storage rounding
    nx, nz = s.grid_v.shape
    s_max = float(np.max(1.0 / s.grid_v.astype(np.float64)))
    bound = (nx + nz) * EPS_SHIFT * s.grid_h * s_max + 0.5 * fp32_ulp(ref.T)
    err = np.abs(T - ref.T)
    assert np.all(err <= bound)
    assert np.max(err) < 1e-7


CASES = [
    # seed, ntr, nx, nz, nt, m, weight, aperture, taper
    (1, 80, 70, 53, 400, 4, "one", 0.0, 0.0),
    (2, 90, 45, 70, 350, 2, "obliq", 0.0, 0.0),
    (3, 70, 40, 33, 300, 1, "obliq", 150.0, 0.0),
    (4, 100, 66, 48, 420, 4, "one", 180.0, 0.3),
]


@pytest.mark.parametrize("case", CASES, ids=[f"m{c[5]}-{c[6]}-A{int(c[7])}-t{c[8]}" for c in CASES])
@pytest.mark.parametrize("pairs", [1, 0])
def test_migrate_matches_oracle(case, pairs):
    seed, ntr, nx, nz, nt, m, weight, ap, taper = case
    s = sv.vxz_model(snapped_survey(seed, ntr, nx, nz, nt, weight=weight, aperture=ap, taper=taper), m,
                     lens_dv=-400.0, lens_r=120.0)
    d = sv.random_traces(s, 9 + seed, smooth=5)
    p = kh.Plan(s)
    p.set_option(kh.KH_OPT_SAMPLE_PAIRS, pairs)
    got, _ = gpu_migrate(s, d, plan=p)
    want = oracle.migrate(s, d)
    assert np.count_nonzero(want) > want.size // 4
    assert rel_l2(got, want) < FP32_REL_L2


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_mixed_traces(dtype):
    s = sv.vxz_model(snapped_survey(5, 90, 64, 48, 400), 4, lens_dv=-400.0, lens_r=120.0)
    d = sv.random_traces(s, 4, smooth=5)
    q = torch.as_tensor(d).to(dtype).float().numpy()
    got, _ = gpu_migrate(s, d, trace_dtype=dtype)
    assert rel_l2(got, oracle.migrate(s, q)) < FP32_REL_L2
    assert rel_l2(got, oracle.migrate(s, d)) < MIXED_REL_L2


def test_line_survey_sampled_points():
    # the 2.5D line geometry (shots every 25 m, split spreads at 12.5 m) with a lens model: the
    # full image against the oracle at sampled points
    s = sv.vxz_model(sv.survey_25d_lsm(nx=160, nz=120, nt=1000, n_shots=10), 4, lens_dv=-350.0, lens_r=150.0)
    sc = sv.reflectors_2d(np.random.default_rng(sv.BASE_SEED), s, spacing=10.0)
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0).numpy()
    got, p = gpu_migrate(s, d)
    rng = np.random.default_rng(3)
    idx = rng.choice(got.size, 3000, replace=False)
    want = oracle.migrate_points(s, d, idx)
    assert np.count_nonzero(want) > 1000
    assert rel_l2(got.ravel()[idx], want) < FP32_REL_L2


def test_lens_diffractor_focuses_with_the_tables():
    s0 = sv.survey_2d_const().replace(vel="linear", v0=1800.0, k=0.5, nz=112)
    s = sv.vxz_model(s0, 2, lens_dv=-450.0, lens_xz=(640.0, 420.0), lens_r=140.0)
    sc = np.array([[640.0, 0.0, 800.0, 1.0]])
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0).numpy()
    got, _ = gpu_migrate(s, d)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2
    stack = got.sum(axis=0)[0]
    px, pz = np.unravel_index(np.argmax(np.abs(stack)), stack.shape)
    assert abs(px - 64) <= 1 and abs(pz - 80) <= 1
    # the background v(z) model ignores the lens: its image of the same data peaks lower
    bg, _ = gpu_migrate(s0, d)
    assert np.max(np.abs(bg.sum(axis=0)[0])) < 0.8 * np.max(np.abs(stack))


def test_missing_location_is_reported_and_skipped():
    s = sv.vxz_model(snapped_survey(6, 60, 40, 40, 300), 4)
    d = sv.random_traces(s, 2, smooth=5)
    loc = kh.locations(s)
    gone = float(s.sx[0])
    keep_loc = loc[loc != np.float32(gone)]
    p = kh.Plan(s.replace(grid_v=None))
    p.set_grid(s.grid_v, s.grid_ox, s.grid_h, keep_loc)
    hdr = kh.Headers.of(s)
    img = p.migrate(hdr, torch.as_tensor(d, device="cuda"))
    with pytest.raises(kh.KirchhoffError) as ei:
        p.sync()
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
    keep = np.flatnonzero((s.sx != np.float32(gone)) & (s.rx != np.float32(gone)))
    sub = s.subset(keep)
    assert rel_l2(img.double().cpu().numpy(), oracle.migrate(sub, d[keep])) < FP32_REL_L2
    p.sync()   # the status was cleared by the report


def test_refusals():
    s = sv.vxz_model(snapped_survey(7, 30, 30, 30, 200), 2)
    d = kh.desc_from(s)
    p = kh.Plan(s.replace(grid_v=None))
    hdr = kh.Headers.of(s)
    tr = torch.zeros((s.ntr, s.nt), device="cuda")
    with pytest.raises(kh.KirchhoffError):               # no tables yet
        p.migrate(hdr, tr)
    v = torch.as_tensor(s.grid_v, device="cuda")
    loc = torch.as_tensor(kh.locations(s), device="cuda")
    G = kh.kh_grid(s.grid_v.shape[0], s.grid_v.shape[1], s.grid_ox, s.grid_h)
    bad = [
        kh.kh_grid(G.nx, G.nz, G.ox, G.h * 1.5),                  # h not 1, 2 or 4 times dz
        kh.kh_grid(G.nx, G.nz - 5, G.ox, G.h),                    # too few rows for the image depths
        kh.kh_grid(G.nx, G.nz, G.ox + 3 * s.dx * 10, G.h),        # image columns not covered
        kh.kh_grid(400, 100, G.ox, G.h),                          # above the node limit
    ]
    for g in bad:
        with pytest.raises(kh.KirchhoffError):
            kh.kirchhoff_grid_tables(p.handle, g, torch.zeros(g.nx * g.nz, device="cuda") + 2000.0, loc.numel(), loc)
    with pytest.raises(kh.KirchhoffError):               # v <= 0
        kh.kirchhoff_grid_tables(p.handle, G, v * 0.0, loc.numel(), loc)
    with pytest.raises(kh.KirchhoffError):               # locations not increasing
        kh.kirchhoff_grid_tables(p.handle, G, v, loc.numel(), loc.flip(0).contiguous())
    far = loc.clone()
    far[-1] = float(G.ox + G.h * G.nx + 10.0)
    with pytest.raises(kh.KirchhoffError):               # a location outside the columns
        kh.kirchhoff_grid_tables(p.handle, G, v, loc.numel(), far)
    p.set_grid(s.grid_v, s.grid_ox, s.grid_h, kh.locations(s))
    with pytest.raises(kh.KirchhoffError) as ei:
        p.demigrate(hdr, torch.zeros(p.image_shape, device="cuda"))
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    with pytest.raises(kh.KirchhoffError):
        kh.Plan(s.replace(dim=3, ny=4))
