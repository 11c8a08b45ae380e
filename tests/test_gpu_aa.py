"""Operator anti-aliasing (``aa_spacing`` > 0; constant velocity and v0 + k z) on the GPU against
the FP64 oracle: migration of random 2D and 3D surveys element by element with every weight (W = 1,
the obliquity weight, the true-amplitude weight at constant velocity), with and without an
aperture taper, fast and exact square roots, sample pairs on and off; demigration and the
dot-product identity between the two CUDA operators with the weight on; the allocation-free entry
point with the weight on; and the refusals (tables, time migration and gridded models, 16-bit
traces with v0 + k z, the batched launch, the velocity gradient)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, gpu_demigrate, gpu_migrate, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu

CASES = [
    # dim, ntr, nx, ny, nz, nt, aperture, taper, spacing (m)
    (3, 90, 19, 21, 35, 260, 0.0, 0.0, 12.5),
    (3, 120, 33, 17, 20, 300, 150.0, 0.25, 25.0),
    (2, 80, 70, 1, 53, 300, 0.0, 0.0, 12.5),
    (2, 70, 45, 1, 40, 257, 120.0, 0.4, 30.0),
]


def aa_survey(case, seed, weight="one", vel="const"):
    dim, ntr, nx, ny, nz, nt, ap, taper, spacing = case
    rng = np.random.default_rng(seed)
    kw = dict(v0=1900.0) if vel == "const" else dict(vel="linear", v0=1600.0, k=0.6)
    s = sv.survey_random(rng, dim, ntr, nx, ny, nz, nt, weight=weight, aperture=ap, n_bins=3, h=12.5, **kw)
    return s.replace(taper=taper, aa_spacing=spacing)


def branch_mix(s):
    """Fraction of (image point, trace) pairs of the survey in each branch of the weight (kept,
    tapered, removed), from the oracle on a sample: the cases must exercise all three."""
    rng = np.random.default_rng(0)
    n = 4000
    ix, iy, iz = rng.integers(0, s.nx, n), rng.integers(0, s.ny, n), rng.integers(1, s.nz, n)
    j = rng.integers(0, s.ntr, n)
    pts = np.stack([s.ox + ix * s.dx, (s.oy + iy * s.dy) if s.dim == 3 else np.zeros(n), s.oz + iz * s.dz,
                    s.sx[j], s.sy[j], s.rx[j], s.ry[j]], 1).astype(np.float64)
    w = oracle.aa_weight(s, pts)
    return np.mean(w == 1.0), np.mean((w > 0) & (w < 1)), np.mean(w == 0.0)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-A{int(c[6])}-t{c[7]}" for c in CASES])
@pytest.mark.parametrize("weight", ["one", "obliq", "ta"])
@pytest.mark.parametrize("fast_math", [True, False])
@pytest.mark.parametrize("pairs", [1, 0])
def test_migrate_matches_oracle(case, weight, fast_math, pairs):
    s = aa_survey(case, 700 + case[1], weight)
    kept, tapered, removed = branch_mix(s)
    assert min(kept, tapered, removed) > 0.02, (kept, tapered, removed)
    d = sv.random_traces(s, 7, smooth=5)
    p = kh.Plan(s, fast_math=fast_math)
    p.set_option(kh.KH_OPT_SAMPLE_PAIRS, pairs)
    got, _ = gpu_migrate(s, d, plan=p)
    want = oracle.migrate(s, d)
    assert np.count_nonzero(want) > 0
    assert rel_l2(got, want) < FP32_REL_L2
    # the weight acts: without it the image differs by far more than the bar
    assert rel_l2(oracle.migrate(s.replace(aa_spacing=0.0), d), want) > 100 * FP32_REL_L2


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-A{int(c[6])}-t{c[7]}" for c in CASES])
@pytest.mark.parametrize("weight", ["one", "obliq"])
@pytest.mark.parametrize("fast_math", [True, False])
@pytest.mark.parametrize("pairs", [1, 0])
def test_migrate_linear_vz_matches_oracle(case, weight, fast_math, pairs):
    s = aa_survey(case, 1700 + case[1], weight, vel="linear")
    kept, tapered, removed = branch_mix(s)
    assert min(kept, tapered, removed) > 0.02, (kept, tapered, removed)
    d = sv.random_traces(s, 9, smooth=5)
    p = kh.Plan(s, fast_math=fast_math)
    p.set_option(kh.KH_OPT_SAMPLE_PAIRS, pairs)
    got, _ = gpu_migrate(s, d, plan=p)
    want = oracle.migrate(s, d)
    assert rel_l2(got, want) < FP32_REL_L2
    assert rel_l2(oracle.migrate(s.replace(aa_spacing=0.0), d), want) > 100 * FP32_REL_L2


@pytest.mark.parametrize("case", CASES[1:3], ids=["3d", "2d"])
@pytest.mark.parametrize("weight,vel", [("one", "const"), ("ta", "const"), ("obliq", "linear")])
def test_demigrate_and_dot_product(case, weight, vel):
    s = aa_survey(case, 900 + case[1], weight, vel)
    d = sv.random_traces(s, 11, smooth=3)
    mc = oracle.migrate(s, d).astype(np.float32)   # a coherent image (see the true-amplitude tests)
    got, p = gpu_demigrate(s, mc)
    assert rel_l2(got, oracle.demigrate(s, mc)) < FP32_REL_L2
    m = sv.random_image(s, 2)
    Ltm, _ = gpu_demigrate(s, m, plan=p)
    Ld, _ = gpu_migrate(s, d, plan=p)
    lhs = float(np.vdot(Ld, m.astype(np.float64)))
    rhs = float(np.vdot(d.astype(np.float64), Ltm))
    # relative to |L d| |m|, the bound of either side: with the weight removing most steep
    # contributions a random image can be nearly orthogonal to L d (on the 2D v(z) line here
    # <L d, m> is 1.3e-5 of |L d| |m|), and the sides' FP32 rounding is not small against the dot
    # itself; leaving the weight out of one operator moves the dot by ~3e-3 of the bound
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(Ld) * np.linalg.norm(m.astype(np.float64))


def test_allocation_free_entry_point():
    s = aa_survey(CASES[0], 41)
    d = sv.random_traces(s, 3, smooth=5)
    hdr = kh.Headers.of(s)
    img = torch.full(tuple(int(v) for v in s.image_shape), float("nan"), device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    kh.kirchhoff_migrate_noalloc(kh.desc_from(s), hdr.ntr, *hdr.args(), torch.as_tensor(d, device="cuda"), img,
                                 status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert rel_l2(img.double().cpu().numpy(), oracle.migrate(s, d)) < FP32_REL_L2


def test_zero_spacing_is_the_plain_operator():
    s = aa_survey(CASES[1], 43)
    d = sv.random_traces(s, 5, smooth=5)
    a, _ = gpu_migrate(s.replace(aa_spacing=0.0), d)
    b, _ = gpu_migrate(s.replace(aa_spacing=0.0, taper=0.0), d)
    assert rel_l2(a, oracle.migrate(s.replace(aa_spacing=0.0), d)) < FP32_REL_L2
    assert rel_l2(b, oracle.migrate(s.replace(aa_spacing=0.0, taper=0.0), d)) < FP32_REL_L2


def test_refusals():
    rng = np.random.default_rng(3)
    s = sv.survey_random(rng, 3, 20, 8, 8, 16, 64).replace(aa_spacing=12.5)
    for bad in (s.replace(vel="pstm", oz=0.0, dz=0.008), s.replace(vel="table"), s.replace(aa_spacing=-1.0),
                s.replace(aa_spacing=float("inf"))):
        with pytest.raises(kh.KirchhoffError) as ei:
            kh.Plan(bad)
        want = kh.KH_ERR_UNSUPPORTED if bad.aa_spacing > 0 and np.isfinite(bad.aa_spacing) else kh.KH_ERR_INVALID_ARG
        assert ei.value.status == want
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Plan(s.replace(vel="linear", k=0.5), trace_dtype=torch.float16)
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    p = kh.Plan(s)
    hdr = kh.Headers.of(s)
    with pytest.raises(kh.KirchhoffError) as ei:
        p.velocity_grad(hdr, torch.zeros(p.image_shape, device="cuda"), torch.zeros((s.ntr, s.nt), device="cuda"))
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Batch([(p, hdr, torch.zeros((s.ntr, s.nt), device="cuda"), torch.zeros(p.image_shape, device="cuda"))])
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
