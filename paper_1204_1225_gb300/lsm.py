"""Differentiable migration operators and least-squares migration.

``KirchhoffMigrate`` (image = L(v0, k) traces, Eq. 1) and ``KirchhoffDemigrate``
(traces = L(v0, k)^T image) are torch.autograd.Functions whose backward passes run the
library's adjoint kernel and its (v0, k) gradient kernel:

    migrate:    d<g, L d>/d d = L^T g,   d<g, L d>/d(v0, k) = velocity_grad(m=g, D=d)
    demigrate:  d<g, L^T m>/d m = L g,   d<g, L^T m>/d(v0, k) = velocity_grad(m=m, D=g)

``cgls`` solves min_m ||L^T m - d||^2 (least-squares migration; the demigration is the
modelling operator) with the textbook CGLS recursion, FP64 inner products and an optional
on-disk checkpoint of the iterate state so that a run can resume.  ``lsm_descent`` is the
same objective minimised through autograd, one checkpointed graph per iteration.
"""
from __future__ import annotations

import os
from typing import Dict, Optional, Tuple

import torch
import torch.utils.checkpoint

from . import kirchhoff as kh


class Operator:
    """The migration operator of one survey geometry; plans are cached per (v0, k)."""

    def __init__(self, survey, device="cuda", fast_math: bool = True):
        self.survey = survey
        self.device = torch.device(device)
        self.hdr = kh.Headers.of(survey, device=self.device)
        self.fast_math = fast_math
        self._plans: Dict[Tuple[float, float], kh.Plan] = {}
        self.image_shape = (survey.n_bins, survey.ny if survey.dim == 3 else 1, survey.nx, survey.nz)
        self.trace_shape = (survey.ntr, survey.nt)

    def plan(self, v0: Optional[float] = None, k: Optional[float] = None) -> kh.Plan:
        v0 = float(self.survey.v0 if v0 is None else v0)
        k = float(self.survey.k if k is None else k)
        key = (v0, k)
        p = self._plans.get(key)
        if p is None:
            p = kh.Plan(self.survey.replace(v0=v0, k=k), fast_math=self.fast_math)
            self._plans[key] = p
        return p

    def L(self, traces, v0=None, k=None):
        return self.plan(v0, k).migrate(self.hdr, traces.contiguous())

    def LT(self, image, v0=None, k=None):
        return self.plan(v0, k).demigrate(self.hdr, image.contiguous())

    def vgrad(self, image, traces, v0=None, k=None):
        return self.plan(v0, k).velocity_grad(self.hdr, image.contiguous(), traces.contiguous())


def _scalar(x):
    return float(x.item()) if torch.is_tensor(x) else float(x)


class KirchhoffMigrate(torch.autograd.Function):
    """image = L(v0, k) traces (Eq. 1)."""

    @staticmethod
    def forward(ctx, traces, v0, k, op: Operator):
        ctx.op = op
        ctx.vk = (_scalar(v0), _scalar(k))
        ctx.save_for_backward(traces)
        ctx.vk_tensors = (torch.is_tensor(v0), torch.is_tensor(k))
        return op.L(traces, *ctx.vk)

    @staticmethod
    def backward(ctx, g):
        (traces,) = ctx.saved_tensors
        op = ctx.op
        g = g.contiguous()
        gd = op.LT(g, *ctx.vk) if ctx.needs_input_grad[0] else None
        gv = gk = None
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            gvk = op.vgrad(g, traces, *ctx.vk)
            gv, gk = gvk[0], gvk[1]
        return gd, gv, gk, None


class KirchhoffDemigrate(torch.autograd.Function):
    """traces = L(v0, k)^T image (the transpose of Eq. 1)."""

    @staticmethod
    def forward(ctx, image, v0, k, op: Operator):
        ctx.op = op
        ctx.vk = (_scalar(v0), _scalar(k))
        ctx.save_for_backward(image)
        return op.LT(image, *ctx.vk)

    @staticmethod
    def backward(ctx, g):
        (image,) = ctx.saved_tensors
        op = ctx.op
        g = g.contiguous()
        gm = op.L(g, *ctx.vk) if ctx.needs_input_grad[0] else None
        gv = gk = None
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            gvk = op.vgrad(image, g, *ctx.vk)
            gv, gk = gvk[0], gvk[1]
        return gm, gv, gk, None


def migrate(traces, v0, k, op: Operator):
    return KirchhoffMigrate.apply(traces, v0, k, op)


def demigrate(image, v0, k, op: Operator):
    return KirchhoffDemigrate.apply(image, v0, k, op)


def _dot(a, b) -> float:
    return float(torch.dot(a.reshape(-1).double(), b.reshape(-1).double()).item())


def cgls(op: Operator, data, n_iter: int = 20, m0=None, checkpoint: Optional[str] = None,
         resume: bool = False, v0=None, k=None):
    """CGLS for min_m ||L^T m - d||^2 in FP32 vectors with FP64 inner products.

    Returns (m, residual norms ||r_i||, normal-residual norms ||L r_i||).  With
    ``checkpoint`` the iterate state (m, r, s, p, gamma, iteration, histories) is saved after
    every iteration; ``resume=True`` continues from that file.
    """
    d = data.contiguous()
    state = None
    if resume and checkpoint and os.path.exists(checkpoint):
        state = torch.load(checkpoint, map_location=op.device)
    if state is None:
        m = torch.zeros(op.image_shape, device=op.device) if m0 is None else m0.clone()
        r = d.clone() if m0 is None else d - op.LT(m, v0, k)
        s = op.L(r, v0, k)
        state = {"m": m, "r": r, "s": s, "p": s.clone(), "gamma": _dot(s, s), "it": 0,
                 "rn": [float(torch.linalg.vector_norm(r.double()))], "sn": [_dot(s, s) ** 0.5]}
    m, r, s, p, gamma = state["m"], state["r"], state["s"], state["p"], state["gamma"]
    while state["it"] < n_iter:
        q = op.LT(p, v0, k)
        qq = _dot(q, q)
        if qq == 0.0 or gamma == 0.0:
            break
        alpha = gamma / qq
        m.add_(p, alpha=alpha)
        r.add_(q, alpha=-alpha)
        s = op.L(r, v0, k)
        gamma_new = _dot(s, s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        state.update(m=m, r=r, s=s, p=p, gamma=gamma, it=state["it"] + 1)
        state["rn"].append(float(torch.linalg.vector_norm(r.double())))
        state["sn"].append(gamma ** 0.5)
        if checkpoint:
            tmp = checkpoint + ".tmp"
            torch.save(state, tmp)
            os.replace(tmp, checkpoint)
    return m, torch.tensor(state["rn"], dtype=torch.float64), torch.tensor(state["sn"], dtype=torch.float64)


def lsm_descent(op: Operator, data, n_iter: int = 5, m0=None, use_checkpoint: bool = True):
    """Steepest descent on J(m) = 1/2 ||L^T m - d||^2 through autograd (the backward pass
    runs the migration kernel), with the exact step for a quadratic, ||g||^2 / ||L^T g||^2.
    Each iteration's graph is wrapped in torch.utils.checkpoint so only the image is kept."""
    m = torch.zeros(op.image_shape, device=op.device) if m0 is None else m0.clone()
    v0 = torch.tensor(op.survey.v0, dtype=torch.float64)
    k = torch.tensor(op.survey.k, dtype=torch.float64)
    losses = []

    def objective(mm):
        res = KirchhoffDemigrate.apply(mm, v0, k, op) - data
        return 0.5 * torch.sum(res.double() ** 2)

    for _ in range(n_iter):
        mm = m.detach().requires_grad_(True)
        if use_checkpoint:
            J = torch.utils.checkpoint.checkpoint(objective, mm, use_reentrant=False)
        else:
            J = objective(mm)
        J.backward()
        g = mm.grad.detach()
        Lg = op.LT(g)
        step = _dot(g, g) / max(_dot(Lg, Lg), 1e-300)
        m = (m - step * g).detach()
        losses.append(float(J.item()))
    return m, losses
