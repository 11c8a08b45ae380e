"""Host-resident migration (kirchhoff_migrate_host): inputs in host memory, the image back in host
memory, consecutive calls pipelined over two slots of device buffers and two copy streams.  Every
image equals the device entry point's bit for bit (and the FP64 oracle's within the FP32 bar),
with several calls in flight on different inputs, a growing trace count, pageable buffers, 16-bit
traces and 2D surveys; the refusals."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu


def _survey(seed, ntr, dim=3):
    rng = np.random.default_rng(seed)
    return sv.survey_random(rng, dim, ntr, 21, 17 if dim == 3 else 1, 36, 300, vel="linear", weight="obliq",
                            aperture=160.0, n_bins=3, h=12.5, v0=1700.0, k=0.5)


def _host_inputs(s, seed, dtype=torch.float32, pin=True):
    d = torch.as_tensor(sv.random_traces(s, seed, smooth=5)).to(dtype)
    hdr = [torch.as_tensor(a, dtype=torch.float32) for a in (s.sx, s.sy, s.rx, s.ry)]
    if pin:
        d = d.pin_memory()
        hdr = [t.pin_memory() for t in hdr]
    return hdr, d


def _device_image(plan, hdr, d):
    img = plan.migrate(kh.Headers(*hdr, device="cuda"), d.to("cuda"))
    plan.sync()
    return img.cpu()


@pytest.mark.parametrize("dim", [3, 2])
def test_pipelined_calls_match_the_device_entry_point(dim):
    s = _survey(11, 400, dim)
    plan = kh.Plan(s)
    inputs = [_host_inputs(s, 20 + i) for i in range(5)]
    outs = [torch.full(plan.image_shape, float("nan")).pin_memory() for _ in inputs]
    for (hdr, d), out in zip(inputs, outs):   # five calls enqueued back to back
        plan.migrate_host(hdr, d, out)
    plan.host_join()
    plan.sync()
    for (hdr, d), out in zip(inputs, outs):
        assert torch.equal(out, _device_image(plan, hdr, d))
    hdr, d = inputs[0]
    assert rel_l2(outs[0].double().numpy(), oracle.migrate(s, d.double().numpy())) < FP32_REL_L2


def test_trace_count_grows_and_pageable_buffers():
    small, large = _survey(12, 150), _survey(13, 900)
    plan = kh.Plan(large)
    seq = [(small, True), (large, True), (small, False), (large, False)]
    res = []
    for i, (s, pin) in enumerate(seq):
        hdr, d = _host_inputs(s, 40 + i, pin=pin)
        out = torch.empty(plan.image_shape)
        if pin:
            out = out.pin_memory()
        plan.migrate_host(hdr, d, out)
        res.append((hdr, d, out))
    plan.host_join()
    plan.sync()
    for hdr, d, out in res:
        assert torch.equal(out, _device_image(plan, hdr, d))


def test_half_precision_traces():
    s = _survey(14, 300)
    plan = kh.Plan(s, trace_dtype=torch.float16)
    hdr, d = _host_inputs(s, 5, dtype=torch.float16)
    out = torch.empty(plan.image_shape).pin_memory()
    plan.migrate_host(hdr, d, out)
    plan.host_join()
    plan.sync()
    assert torch.equal(out, _device_image(plan, hdr, d))


def test_refusals():
    s = _survey(15, 50)
    plan = kh.Plan(s)
    hdr, d = _host_inputs(s, 1, pin=False)
    out = torch.empty(plan.image_shape)
    with pytest.raises(ValueError):
        plan.migrate_host(hdr, d.cuda(), out)                 # device traces
    with pytest.raises(ValueError):
        plan.migrate_host(hdr, d, out.cuda())                 # device image
    with pytest.raises(ValueError):
        plan.migrate_host(hdr, d[:-1], out)                   # short traces
    with pytest.raises(ValueError):
        plan.migrate_host(hdr, d.double(), out)               # wrong dtype
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.kirchhoff_migrate_host(plan.handle, s.ntr, *hdr, d, None)
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
    with pytest.raises(kh.KirchhoffError) as ei:
        kh.kirchhoff_migrate_host(plan.handle, -1, *hdr, d, out)
    assert ei.value.status == kh.KH_ERR_INVALID_ARG
