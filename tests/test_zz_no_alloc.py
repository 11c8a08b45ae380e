"""The allocation-free migration entry point (for callers that cannot allocate device memory:
their HBM belongs to another allocator's pool, or they must not call cudaMalloc after start-up
because it can synchronise the device).  It must give the plan path's result, call after call,
although its fixed scratch keeps the previous call's contents.  Collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv


def _survey(seed, ntr, nb):
    rng = np.random.default_rng(seed)
    return sv.survey_random(rng, 3, ntr, 22, 19, 40, 320, vel="linear", weight="obliq",
                            aperture=150.0, n_bins=nb, h=12.5, v0=1600.0, k=0.6, t0=0.004)


@pytest.mark.gpu
def test_noalloc_matches_plan_path_on_consecutive_calls():
    # a large survey first, then a smaller one with fewer bins: stale scratch must not leak
    for seed, ntr, nb in ((31, 3000, 5), (32, 700, 3)):
        s = _survey(seed, ntr, nb)
        d = torch.as_tensor(sv.random_traces(s, seed, smooth=5), device="cuda")
        hdr = kh.Headers.of(s)
        plan = kh.Plan(s)
        want = plan.migrate(hdr, d)
        plan.sync()
        got = torch.full(plan.image_shape, float("nan"), device="cuda")
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        kh.kirchhoff_migrate_noalloc(kh.desc_from(s), hdr.ntr, *hdr.args(), d, got, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert rel_l2(got.double().cpu().numpy(), want.double().cpu().numpy()) <= FP32_REL_L2
        # and against the FP64 oracle directly
        assert rel_l2(got.double().cpu().numpy(), oracle.migrate(s, d.cpu().numpy())) < FP32_REL_L2


def test_noalloc_rejects_inputs_beyond_its_scratch():
    s = _survey(33, 10, 2)
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.lib()
        import ctypes
        rc = kh.lib().kirchhoff_migrate_noalloc(ctypes.byref(kh.desc_from(s)), 65537, None, None,
                                                None, None, None, None, None, None)
        kh._check(rc)
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
    assert "65536" in str(ei.value)
