"""Mixed precision: traces stored as FP16 or BF16 in HBM and in the shared-memory ring,
interpolation and accumulation in FP32.  The kernel must match the FP64 oracle fed the same
16-bit sample values (the same algorithm) at the FP32 bar, and the image error caused by the
16-bit storage itself must stay within the mixed-precision bar."""
import numpy as np
import pytest
import torch

import oracle
from helpers import (FP32_REL_L2, MIXED_REL_L2, cfg1_inputs, cfg2_reduced, cfg4_reduced,
                     gpu_migrate, quantize, rel_l2)

pytestmark = pytest.mark.gpu

INPUTS = {"2d-const": cfg1_inputs, "3d-vz": cfg2_reduced, "25d-vz": cfg4_reduced}


@pytest.mark.parametrize("name", sorted(INPUTS))
@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16], ids=["f16", "bf16"])
def test_16bit_traces(name, dtype):
    s, d = INPUTS[name]()
    got, _ = gpu_migrate(s, d, trace_dtype=dtype)
    same_algorithm = oracle.migrate(s, quantize(d, dtype))
    exact = oracle.migrate(s, d)
    e_same = rel_l2(got, same_algorithm)
    err = rel_l2(got, exact)
    print(f"{name} {dtype}: vs same-algorithm oracle {e_same:.2e}, vs FP32-data oracle {err:.2e}")
    assert e_same < FP32_REL_L2
    assert err < MIXED_REL_L2, err
