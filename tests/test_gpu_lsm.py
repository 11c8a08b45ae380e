"""Autograd Functions over the CUDA operators and least-squares migration (CGLS with FP64
inner products, checkpoint / resume), checked against the FP64 oracle."""
import os

import numpy as np
import pytest
import torch

import oracle
from helpers import FP32_REL_L2, GRAD_REL, rel_l2
from paper_1204_1225_gb300 import lsm
from paper_1204_1225_gb300 import survey as sv

pytestmark = pytest.mark.gpu


def small_25d():
    return sv.survey_25d_lsm(nx=64, nz=50, nt=400, n_shots=8, n_rec=40)


def test_autograd_migrate_gradients():
    s = small_25d()
    op = lsm.Operator(s)
    d = torch.as_tensor(sv.random_traces(s, 1, smooth=9), device="cuda").requires_grad_(True)
    m = torch.as_tensor(sv.random_image(s, 2), device="cuda")
    v0 = torch.tensor(s.v0, dtype=torch.float64, requires_grad=True)
    k = torch.tensor(s.k, dtype=torch.float64, requires_grad=True)
    img = lsm.migrate(d, v0, k, op)
    assert rel_l2(img.detach().double().cpu().numpy(), oracle.migrate(s, d.detach().cpu().numpy())) < FP32_REL_L2
    torch.sum(img * m).backward()
    # d/dd <m, L d> = L^T m
    assert rel_l2(d.grad.double().cpu().numpy(), oracle.demigrate(s, m.cpu().numpy())) < FP32_REL_L2
    want, scale = oracle.vgrad(s, m.cpu().numpy(), d.detach().cpu().numpy(), return_abs=True)
    assert abs(v0.grad.item() - want[0]) <= GRAD_REL * scale[0]
    assert abs(k.grad.item() - want[1]) <= GRAD_REL * scale[1]


def test_autograd_demigrate_gradients():
    s = small_25d()
    op = lsm.Operator(s)
    m = torch.as_tensor(sv.random_image(s, 3), device="cuda").requires_grad_(True)
    g = torch.as_tensor(sv.random_traces(s, 4, smooth=9), device="cuda")
    v0 = torch.tensor(s.v0, dtype=torch.float64, requires_grad=True)
    k = torch.tensor(s.k, dtype=torch.float64, requires_grad=True)
    tr = lsm.demigrate(m, v0, k, op)
    torch.sum(tr * g).backward()
    # d/dm <g, L^T m> = L g ; d/dth <g, L^T m> = d/dth <L g, m>
    assert rel_l2(m.grad.double().cpu().numpy(), oracle.migrate(s, g.cpu().numpy())) < FP32_REL_L2
    want, scale = oracle.vgrad(s, m.detach().cpu().numpy(), g.cpu().numpy(), return_abs=True)
    assert abs(v0.grad.item() - want[0]) <= GRAD_REL * scale[0]
    assert abs(k.grad.item() - want[1]) <= GRAD_REL * scale[1]


def test_cgls_matches_oracle_and_resumes(tmp_path):
    s = small_25d()
    op = lsm.Operator(s)
    rng = np.random.default_rng(5)
    sc = sv.reflectors_2d(rng, s, n_lines=2, n_diffractors=4, spacing=10.0)
    d_np = sv.synthesize(s, sc, oracle.arrival_times, 25.0, device="cuda").cpu().numpy()
    d = torch.as_tensor(d_np, device="cuda")
    n = 8
    m_gpu, rn_gpu, _ = lsm.cgls(op, d, n_iter=n)
    m_or, rn_or, _ = oracle.cgls(s, d_np, n_iter=n)
    assert np.all(np.diff(rn_gpu.numpy()) <= 1e-6 * rn_gpu[0].item())      # residual decreases
    assert np.allclose(rn_gpu.numpy(), rn_or, rtol=1e-4)
    assert rel_l2(m_gpu.double().cpu().numpy(), m_or) < 1e-3
    # checkpoint after 4 iterations, resume to 8: same iterate as 8 straight iterations
    ck = os.path.join(str(tmp_path), "cgls.pt")
    lsm.cgls(op, d, n_iter=4, checkpoint=ck)
    m_res, rn_res, _ = lsm.cgls(op, d, n_iter=n, checkpoint=ck, resume=True)
    assert torch.equal(m_res, m_gpu)
    assert np.array_equal(rn_res.numpy(), rn_gpu.numpy())


def test_lsm_descent_with_checkpointed_graph_decreases_the_misfit():
    s = small_25d()
    op = lsm.Operator(s)
    d = torch.as_tensor(sv.random_traces(s, 6, smooth=9), device="cuda")
    _, losses = lsm.lsm_descent(op, d, n_iter=4, use_checkpoint=True)
    _, losses_plain = lsm.lsm_descent(op, d, n_iter=4, use_checkpoint=False)
    assert all(b < a for a, b in zip(losses, losses[1:]))
    assert np.allclose(losses, losses_plain, rtol=1e-6)
