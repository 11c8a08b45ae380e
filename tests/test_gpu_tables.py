"""Traveltime tables (mixed precision): the v(z) model read from one radial table T(h, z)
on a 25 m grid, stored as F32, FP16 (per h row, the residual of a quadratic in depth) or 16-bit
fixed point (offset + scale), interpolated bilinearly in FP32.  The kernel is compared with the FP64 oracle that runs the
same algorithm (closed-form nodes, unquantised, same bilinear rule); the error of the table
itself against the closed form is reported, not gated."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, MIXED_REL_L2, cfg1_inputs, cfg2_reduced, gpu_migrate, quantize, rel_l2
from paper_1204_1225_gb300 import kirchhoff as kh

pytestmark = pytest.mark.gpu


def _run(s, d, table_dtype, trace_dtype=torch.float32):
    p = kh.Plan(s, trace_dtype=trace_dtype, table_dtype=table_dtype)
    got, _ = gpu_migrate(s, d, trace_dtype=trace_dtype, plan=p)
    return got


# table storage -> bar against the same-algorithm FP64 oracle: FP32 nodes carry the FP32 bar,
# the 16-bit tables the mixed-precision bar
BARS = {"f32": FP32_REL_L2, "u16": MIXED_REL_L2, "f16": MIXED_REL_L2}


@pytest.mark.parametrize("tdt", ["f32", "u16", "f16"])
def test_table_2d_const(tdt):
    s, d = cfg1_inputs()
    st = s.replace(vel="table", table_spacing=25.0)
    got = _run(st, d, tdt)
    same = oracle.migrate(st, d)
    err = rel_l2(got, same)
    print(f"2d table {tdt}: vs same-algorithm oracle {err:.2e}, "
          f"vs closed-form oracle {rel_l2(got, oracle.migrate(s, d)):.2e}")
    assert err < BARS[tdt]


@pytest.mark.parametrize("tdt", ["f32", "u16", "f16"])
def test_table_3d_vz(tdt):
    s, d = cfg2_reduced()
    st = s.replace(vel="table", table_spacing=25.0)
    got = _run(st, d, tdt)
    same = oracle.migrate(st, d)
    err = rel_l2(got, same)
    print(f"3d table {tdt}: vs same-algorithm oracle {err:.2e}, "
          f"vs closed-form oracle {rel_l2(got, oracle.migrate(s, d)):.2e}")
    assert err < BARS[tdt]


@pytest.mark.parametrize("tdt", ["u16", "f16"])
def test_table_16bit_with_fp16_traces(tdt):
    s, d = cfg2_reduced()
    st = s.replace(vel="table", table_spacing=25.0)
    got = _run(st, d, tdt, trace_dtype=torch.float16)
    assert rel_l2(got, oracle.migrate(st, d)) < MIXED_REL_L2


def test_table_plans_refuse_adjoint_and_gradient():
    s, d = cfg1_inputs()
    p = kh.Plan(s.replace(vel="table"))
    hdr = kh.Headers.of(s)
    m = torch.zeros(p.image_shape, device="cuda")
    with pytest.raises(kh.KirchhoffError) as ei:
        p.demigrate(hdr, m)
    assert ei.value.status == kh.KH_ERR_UNSUPPORTED
