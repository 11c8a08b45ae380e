"""Shared helpers for the GPU parity tests (inputs are seeded; expected values come from
the FP64 oracle only)."""
import numpy as np
import torch

import oracle
from paper_1204_1225_gb300 import survey as sv

# Parity bar of the FP32 path against the FP64 oracle: relative L2 error of the image.
FP32_REL_L2 = 1e-5


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_migrate(s, traces, trace_dtype=torch.float32, fast_math=True, tile=None, plan=None):
    from paper_1204_1225_gb300 import kirchhoff as kh
    p = plan or kh.Plan(s, trace_dtype=trace_dtype, fast_math=fast_math, tile=tile)
    hdr = kh.Headers.of(s)
    d = torch.as_tensor(np.asarray(traces)).to("cuda", trace_dtype).contiguous()
    img = p.migrate(hdr, d)
    p.sync()
    return img.double().cpu().numpy(), p


def cfg1_inputs(noise=0.1):
    s = sv.survey_2d_const()
    sc = sv.point_scatterers_2d(np.random.default_rng(sv.BASE_SEED))
    d = sv.synthesize(s, sc, oracle.arrival_times, 25.0, noise_sigma=noise).numpy()
    return s, d
