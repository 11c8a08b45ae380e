"""Batched persistent launch: many migrations of uneven size in one kernel.

Each job of a batch must produce the image that kirchhoff_migrate produces with the same
plan, bit for bit (same tile computation, same trace order), so the batch inherits the
per-job parity with the oracle; small batches are also compared with the oracle directly.
Covered: ragged grids, padded trace rows, an empty job, jobs of both ln(1 + rho) fit lengths
in one batch, explicit tiles, FP16 traces, CUDA-graph capture and replay with traces changed
in place, refusals, a bounded wait running out, and the tile autotuner."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300.autotune import TileTuner
from paper_1204_1225_gb300.survey import BASE_SEED, random_traces, survey_3d_gradient

pytestmark = pytest.mark.gpu


def _job(s, seed, dtype=torch.float32, tile=None):
    p = kh.Plan(s, trace_dtype=dtype, tile=tile)
    hdr = kh.Headers.of(s)
    d = torch.from_numpy(random_traces(s, seed)).to("cuda").to(dtype).contiguous()
    img = torch.full(p.image_shape, float("nan"), device="cuda")   # every sample must be written
    return p, hdr, d, img


def _small_cube(ntr, n, nt, h=12.5):
    """survey_3d_gradient's geometry with an n^3 image of spacing h centred under the spread."""
    s = survey_3d_gradient(ntr, 256).replace(nt=nt)
    o = 1600.0 - 0.5 * (n - 1) * h
    return s.replace(nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, ox=o, oy=o, name=f"cube{n}-{ntr}tr")


def _per_job(jobs):
    return [p.migrate(h, d) for (p, h, d, _) in jobs]


def _specs():
    # (survey, tile): ragged grids, nt not a multiple of 4 (padded rows), an empty job, a
    # 20-term fit (48^3 at 66.7 m) beside 12-term ones, explicit tiles
    return [
        (survey_3d_gradient(700, 48).replace(nt=601), None),
        (survey_3d_gradient(1500, 96).replace(nt=1000), None),
        (_small_cube(300, 33, 750), None),
        (_small_cube(0, 40, 500), None),
        (_small_cube(900, 50, 803), (16, 8, 2)),
        (survey_3d_gradient(1200, 64).replace(nt=900), (32, 8, 1)),
    ]


@pytest.mark.parametrize("mode", ["persistent", "concurrent"])
def test_batched_equals_per_job_fp32(mode):
    jobs = [_job(s, BASE_SEED + i, tile=t) for i, (s, t) in enumerate(_specs())]
    b = kh.Batch(jobs, mode=mode)
    info = b.info()
    assert info["items"] > 0 and (mode == "concurrent" or 0 < info["ctas"] <= info["items"])
    b.run()
    b.sync()
    ref = _per_job(jobs)
    for i, ((p, h, d, img), r) in enumerate(zip(jobs, ref)):
        assert torch.equal(img, r), f"job {i}: batched image differs from kirchhoff_migrate"
    assert torch.count_nonzero(jobs[3][3]) == 0   # the empty job writes zeros
    b.close()


def test_batched_vs_oracle():
    specs = [(_small_cube(250, 24, 700), None), (_small_cube(400, 32, 750), (16, 8, 2)),
             (_small_cube(150, 20, 601), None)]
    jobs = [_job(s, BASE_SEED + 10 + i, tile=t) for i, (s, t) in enumerate(specs)]
    b = kh.Batch(jobs)
    b.run()
    b.sync()
    for (s, _), (p, h, d, img) in zip(specs, jobs):
        want = oracle.migrate(s, d.cpu().numpy())
        err = rel_l2(img.cpu(), want)
        print(f"{s.name}: rel L2 vs oracle {err:.2e}")
        assert err < FP32_REL_L2


@pytest.mark.parametrize("mode", ["persistent", "concurrent"])
def test_batched_graph_replay_reads_traces_in_place(mode):
    jobs = [_job(s, BASE_SEED + 20 + i, tile=t) for i, (s, t) in enumerate(_specs()[:3])]
    b = kh.Batch(jobs, mode=mode)
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    first = [img.clone() for (_, _, _, img) in jobs]
    for (p, h, d, img), r in zip(jobs, _per_job(jobs)):
        assert torch.equal(img, r)
    for (_, _, d, _) in jobs:
        d.mul_(2.0)
    b.replay()
    b.sync()
    for (_, _, _, img), f in zip(jobs, first):
        assert torch.equal(img, 2.0 * f)   # x2 is exact in FP32 at every step
    b.close()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("mode", ["persistent", "concurrent"])
def test_batched_16bit_traces(dtype, mode):
    specs = [(survey_3d_gradient(800, 64).replace(nt=1001), None), (_small_cube(500, 40, 750), None)]
    jobs = [_job(s, BASE_SEED + 30 + i, dtype=dtype, tile=t) for i, (s, t) in enumerate(specs)]
    b = kh.Batch(jobs, mode=mode)
    b.run()
    b.sync()
    for (p, h, d, img), r in zip(jobs, _per_job(jobs)):
        assert torch.equal(img, r)


def test_batched_refusals():
    s = _small_cube(100, 24, 500)
    a = _job(s, 1)
    c = _job(s.replace(k=0.0), 2)            # constant velocity next to linear v(z)
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Batch([a, c])
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    f16 = _job(s, 3, dtype=torch.float16)   # mixed trace dtypes
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Batch([a, f16])
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    t = _job(s.replace(vel="table"), 4)      # tables are not batched
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.Batch([t])
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.kirchhoff_batched_prepare([])
    assert ei.value.status == kh.KH_ERR_INVALID_ARG


def test_batched_wait_timeout_reports_and_context_survives():
    s = _small_cube(3000, 32, 1500).replace(n_bins=1)   # one bin: many stages per item
    p, h, d, img = _job(s, 5)
    p.set_option(kh.KH_OPT_WAIT_POLLS, 1)
    b = kh.Batch([(p, h, d, img)])
    b.run()
    with pytest.raises(kh.KirchhoffError) as ei:
        b.sync()
    assert ei.value.status == kh.KH_ERR_TIMEOUT
    b.close()
    p.set_option(kh.KH_OPT_WAIT_POLLS, 0)
    b = kh.Batch([(p, h, d, img)])
    b.run()
    b.sync()
    assert torch.equal(img, p.migrate(h, d))


def test_autotuner_picks_a_runnable_tile_and_caches(tmp_path):
    s = survey_3d_gradient(2000, 64).replace(nt=1000)
    p, h, d, img = _job(s, 6)
    tuner = TileTuner(path=str(tmp_path / "tiles.json"), sample_traces=1000, reps=1)
    tile = tuner.choose(p, h, d)
    assert tile in [tuple(c) for c in tuner.candidates[3]]
    assert tuner.timed >= 2
    again = TileTuner(path=str(tmp_path / "tiles.json"))
    assert again.choose(p, h, d) == tile and again.timed == 0
    # the tuned plan still computes the same image as a plan given that tile directly
    q = kh.Plan(s, tile=tile)
    assert torch.equal(p.migrate(h, d), q.migrate(h, d))


@pytest.mark.parametrize("mode", ["persistent", "concurrent"])
def test_batched_constant_velocity_jobs_from_the_batch_generator(mode):
    """The batch workload's own job recipe (constant v, W = 1, full aperture, 8 bins,
    random sources and receivers over the footprint) at small sizes."""
    from paper_1204_1225_gb300.survey import survey_batch_3d
    specs = survey_batch_3d(5, n_range=(17, 40), ntr_range=(50, 400), nt_range=(300, 520))
    jobs = [_job(s, BASE_SEED + 40 + i) for i, s in enumerate(specs)]
    b = kh.Batch(jobs, mode=mode)
    b.run()
    b.sync()
    for (p, h, d, img), r in zip(jobs, _per_job(jobs)):
        assert torch.equal(img, r)
    s, (p, h, d, img) = specs[0], jobs[0]
    err = rel_l2(img.cpu(), oracle.migrate(s, d.cpu().numpy()))
    print(f"{s.name}: rel L2 vs oracle {err:.2e}")
    assert err < FP32_REL_L2
