"""Staging FP32 traces as (d[i], d[i+1] - d[i]) pairs (KH_OPT_SAMPLE_PAIRS, the default) must
leave the migrated image bit-identical to plain-sample staging: the step is the same IEEE
difference the interpolation forms from two samples.  Covered: linear and constant velocity,
both weights, fast and IEEE math, odd nt (source rows not 16-byte multiples, padded pair rows),
the longest trace that still pairs, and the first length that falls back to plain staging; the
paired image is also checked against the oracle."""
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300.survey import BASE_SEED, random_traces, survey_2d_const, survey_3d_gradient

pytestmark = pytest.mark.gpu


def _cube(ntr, n, nt, h=12.5):
    """survey_3d_gradient's geometry with an n^3 image of spacing h centred under the spread."""
    s = survey_3d_gradient(ntr, 256).replace(nt=nt)
    o = 1600.0 - 0.5 * (n - 1) * h
    return s.replace(nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, ox=o, oy=o, name=f"cube{n}-{ntr}tr-{nt}nt")


def _both(s, seed, fast=True):
    d = torch.from_numpy(random_traces(s, seed)).to("cuda").contiguous()
    hdr = kh.Headers.of(s)
    p = kh.Plan(s, fast_math=fast)
    paired = p.migrate(hdr, d)
    p.set_option(kh.KH_OPT_SAMPLE_PAIRS, 0)
    plain = p.migrate(hdr, d)
    torch.cuda.synchronize()
    return d, paired, plain


CASES = [
    ("3d-linear-obliq-odd-nt", lambda: survey_3d_gradient(1500, 48).replace(nt=1001), True),
    ("3d-linear-one", lambda: survey_3d_gradient(1200, 64).replace(nt=900, weight="one"), True),
    ("3d-linear-ieee", lambda: survey_3d_gradient(900, 48).replace(nt=803), False),
    ("3d-const-obliq", lambda: survey_3d_gradient(1000, 40).replace(nt=750, k=0.0), True),
    ("2d-const", lambda: survey_2d_const(), True),
    ("3d-linear-longest-paired", lambda: _cube(300, 32, 2460), True),
    ("3d-linear-plain-above-limit", lambda: _cube(300, 32, 2461), True),
]


@pytest.mark.parametrize("name,make,fast", CASES, ids=[c[0] for c in CASES])
def test_pairs_bit_identical_to_plain_staging(name, make, fast):
    s = make()
    _, paired, plain = _both(s, BASE_SEED + 50, fast)
    assert torch.isfinite(paired).all()
    assert torch.equal(paired, plain), f"{name}: pair staging changed the image"


def test_paired_image_matches_oracle():
    s = _cube(600, 32, 901)
    d, paired, _ = _both(s, BASE_SEED + 51)
    err = rel_l2(paired.cpu(), oracle.migrate(s, d.cpu().numpy()))
    print(f"{s.name}: paired rel L2 vs oracle {err:.2e}")
    assert err < FP32_REL_L2


@pytest.mark.parametrize("mode", ["persistent", "concurrent"])
def test_batched_pairs_match_plain_staging(mode):
    """A batch stages every FP32 job as pairs (each launch); with the option off in the first
    job's plan it stages plain rows.  Both give the per-job images bit for bit."""
    specs = [_cube(400, 32, 801), survey_3d_gradient(700, 48).replace(nt=601), _cube(300, 24, 2460)]
    out = {}
    for pairs in (1, 0):
        jobs = []
        for i, s in enumerate(specs):
            p = kh.Plan(s)
            p.set_option(kh.KH_OPT_SAMPLE_PAIRS, pairs)
            d = torch.from_numpy(random_traces(s, BASE_SEED + 60 + i)).to("cuda").contiguous()
            jobs.append((p, kh.Headers.of(s), d, torch.full(p.image_shape, float("nan"), device="cuda")))
        b = kh.Batch(jobs, mode=mode)
        b.run()
        b.sync()
        out[pairs] = [img.clone() for (_, _, _, img) in jobs]
        ref = [p.migrate(h, d) for (p, h, d, _) in jobs]
        for a, r in zip(out[pairs], ref):
            assert torch.equal(a, r)
        b.close()
    for a, c in zip(out[1], out[0]):
        assert torch.equal(a, c)
