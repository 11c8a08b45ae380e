"""Parity of the CUDA migration with the FP64 oracle on the paper's workload shapes
(seismic reflection data: Ricker events from reflectors and diffractors, Sec. 2-3):
the 3D v(z) survey at reduced image resolution, the 2.5D v(z) line, and the full-size 3D
survey (100 000 traces, 256^3 x 16 bins) at sampled image points in the same launch
configuration the benchmark times."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, cfg2_reduced, cfg4_reduced, gpu_migrate, rel_l2, synth_on_gpu
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fast_math", [True, False])
def test_3d_vz_reduced_full_image(fast_math):
    s, d = cfg2_reduced()
    got, _ = gpu_migrate(s, d, fast_math=fast_math)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2


@pytest.mark.parametrize("fast_math", [True, False])
def test_25d_vz_reduced_full_image(fast_math):
    s, d = cfg4_reduced()
    got, _ = gpu_migrate(s, d, fast_math=fast_math)
    assert rel_l2(got, oracle.migrate(s, d)) < FP32_REL_L2


def test_3d_vz_full_size_sampled_points():
    s = sv.survey_3d_gradient()
    sc = sv.reflectors_3d(np.random.default_rng(sv.BASE_SEED), s, spacing=100.0)
    d = synth_on_gpu(s, sc, 20.0)
    got, p = gpu_migrate(s, d)
    idx = sv.sample_points(s, 4096, seed=sv.BASE_SEED + 2)
    want = oracle.migrate_points(s, d, idx)
    assert rel_l2(got.reshape(-1)[idx], want) < FP32_REL_L2
    # the work count of the same launch (Eq. 2) agrees with the survey geometry's count
    from paper_1204_1225_gb300 import kirchhoff as kh
    assert p.count(kh.Headers.of(s)) > 1.4e12


def test_mixed_precision_full_size_sampled_points():
    """The mixed-precision form at full size (100 000 FP16 traces, U16 radial table, 256^3 x
    16 bins) at sampled image points: against the oracle of the same algorithm (its FP64 table
    on the same nodes, fed the same FP16 sample values) at the mixed bar; the error against the
    exact traveltimes and FP32 data is reported."""
    from helpers import MIXED_REL_L2, quantize
    from paper_1204_1225_gb300 import kirchhoff as kh
    s = sv.survey_3d_gradient()
    sc = sv.reflectors_3d(np.random.default_rng(sv.BASE_SEED), s, spacing=100.0)
    d = synth_on_gpu(s, sc, 20.0)
    st = s.replace(vel="table", table_spacing=25.0)
    p = kh.Plan(st, trace_dtype=torch.float16, table_dtype="u16")
    got, _ = gpu_migrate(st, d, trace_dtype=torch.float16, plan=p)
    idx = sv.sample_points(s, 4096, seed=sv.BASE_SEED + 3)
    g = got.reshape(-1)[idx]
    e_same = rel_l2(g, oracle.migrate_points(st, quantize(d, torch.float16), idx))
    e_exact = rel_l2(g, oracle.migrate_points(s, d, idx))
    print(f"full-size U16 table + FP16 traces: vs same-algorithm oracle {e_same:.2e}, "
          f"vs exact-T FP32-data oracle {e_exact:.2e}")
    assert e_same < MIXED_REL_L2
