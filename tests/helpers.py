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


def synth_on_gpu(s, scatterers, freq, noise=0.0, seed=sv.BASE_SEED):
    """Paper-shaped traces (Ricker events at oracle arrival times) synthesised with torch on
    the GPU; the arrival times come from the FP64 oracle, never from the library."""
    return sv.synthesize(s, scatterers, oracle.arrival_times, freq, noise_sigma=noise, seed=seed,
                         device="cuda").cpu().numpy()


def cfg2_reduced(ntr=2000, n=64):
    """The 3D v(z) survey geometry on a coarser image (n^3 covering the same volume)."""
    s = sv.survey_3d_gradient(ntr=ntr, n=n)
    sc = sv.reflectors_3d(np.random.default_rng(sv.BASE_SEED), s, spacing=100.0)
    return s, synth_on_gpu(s, sc, 20.0)


def cfg4_reduced(n_shots=12, nx=160, nz=120, nt=1000):
    s = sv.survey_25d_lsm(nx=nx, nz=nz, nt=nt, n_shots=n_shots)
    sc = sv.reflectors_2d(np.random.default_rng(sv.BASE_SEED), s, spacing=5.0)
    return s, synth_on_gpu(s, sc, 25.0)


def gpu_demigrate(s, image, fast_math=True, plan=None):
    from paper_1204_1225_gb300 import kirchhoff as kh
    p = plan or kh.Plan(s, fast_math=fast_math)
    hdr = kh.Headers.of(s)
    m = torch.as_tensor(np.asarray(image, dtype=np.float32)).to("cuda").contiguous()
    out = p.demigrate(hdr, m)
    p.sync()
    return out.double().cpu().numpy(), p

# Parity bar for the velocity gradient (a sum of ~1e9 signed FP32 terms per call, carried
# in FP64 per (column, trace)) against the FP64 oracle's analytic gradient.
GRAD_REL = 1e-4


def gpu_vgrad(s, image, traces, fast_math=True, plan=None):
    from paper_1204_1225_gb300 import kirchhoff as kh
    p = plan or kh.Plan(s, fast_math=fast_math)
    hdr = kh.Headers.of(s)
    m = torch.as_tensor(np.asarray(image, dtype=np.float32)).to("cuda").contiguous()
    d = torch.as_tensor(np.asarray(traces, dtype=np.float32)).to("cuda").contiguous()
    out = p.velocity_grad(hdr, m, d)
    p.sync()
    return out.cpu().numpy(), p

# Mixed-precision bar: relative L2 error of the image against the FP64 oracle fed the FP32 traces.
MIXED_REL_L2 = 3e-3


def quantize(traces, dtype):
    """The trace values the kernel sees when they are stored as `dtype` (round to nearest even)."""
    return torch.as_tensor(np.asarray(traces, dtype=np.float32)).to(dtype).to(torch.float64).numpy()
