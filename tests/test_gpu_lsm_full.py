"""Least-squares migration at the full size of the 2.5D line (image 512 x 400 at 5 m, 8 bins,
20 000 traces x 2000 samples, v(z) = 1800 + 0.6 z): one migration L and one demigration L^T
against the FP64 oracle on sampled outputs (image samples one by one, whole trace rows), and 20
CGLS iterations whose residual norm decreases monotonically (CGLS minimises ||L^T m - d|| over
growing Krylov spaces) while the normal-equation residual falls."""
import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, rel_l2, synth_on_gpu
from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import lsm
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def line():
    s = sv.survey_25d_lsm()
    sc = sv.reflectors_2d(np.random.default_rng(sv.BASE_SEED), s, spacing=5.0)
    d = synth_on_gpu(s, sc, 25.0)
    return s, d


def test_full_size_migrate_and_adjoint_sampled(line):
    s, d = line
    p = kh.Plan(s)
    hdr = kh.Headers.of(s)
    dt = torch.as_tensor(d, device="cuda")
    img = p.migrate(hdr, dt)
    p.sync()
    idx = sv.sample_points(s, 4096, seed=sv.BASE_SEED + 5)
    got = img.reshape(-1)[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    assert rel_l2(got, oracle.migrate_points(s, d, idx)) < FP32_REL_L2
    # L^T of the migrated image, whole rows of sampled traces
    m = img.contiguous()
    tr = p.demigrate(hdr, m)
    p.sync()
    rows = np.sort(np.random.default_rng(3).choice(s.ntr, 8, replace=False))
    want = oracle.demigrate(s.subset(rows), m.double().cpu().numpy())
    assert rel_l2(tr[torch.as_tensor(rows, device="cuda")].double().cpu().numpy(), want) < FP32_REL_L2


def test_full_size_cgls_twenty_iterations(line):
    s, d = line
    op = lsm.Operator(s)
    dt = torch.as_tensor(d, device="cuda")
    m, rn, gn = lsm.cgls(op, dt, n_iter=20)
    rn, gn = rn.numpy(), gn.numpy()
    assert rn.size == 21 and torch.isfinite(m).all()
    assert np.all(np.diff(rn) <= 1e-6 * rn[0])          # ||r|| never grows
    assert rn[-1] < 0.9 * rn[0]                         # the data misfit falls
    assert gn[-1] < 0.5 * gn[0]                         # the normal-equation residual falls
