"""Velocity analysis on the GPU (Sec. 2): migrate with the current velocity model v(z) = v0 + k z,
measure how much the redundant offset images disagree, correct (v0, k), migrate again.

The measure is the library's semblance objective (kirchhoff_semblance): the normalised variance
of the weighted offset images across the bins, V(v0, k).  Its gradient comes from the library's
kernels alone: the semblance kernel writes dV/dI, and the velocity-gradient kernel turns it into
dV/d(v0, k) = d<dV/dI, L(v0, k) D>/d(v0, k).  ``VelocityAnalysis.run`` minimises V with a BFGS
iteration on scaled parameters and an Armijo backtracking line search (host logic on two
numbers; every image and gradient is computed on the device).
"""
from __future__ import annotations

import numpy as np
import torch

from . import kirchhoff as kh


class VelocityAnalysis:
    """The velocity-analysis loop for one survey and its traces (device tensors)."""

    def __init__(self, survey, traces, fast_math: bool = True, device="cuda"):
        self.survey = survey
        self.device = torch.device(device)
        self.hdr = kh.Headers.of(survey, device=self.device)
        self.traces = traces.to(self.device, torch.float32).contiguous()
        self.fast_math = fast_math
        self.evaluations = 0

    def objective(self, v0: float, k: float, grad: bool = True):
        """(V, dV/dv0, dV/dk) of the offset images migrated with v(z) = v0 + k z."""
        plan = kh.Plan(self.survey.replace(v0=float(v0), k=float(k)), fast_math=self.fast_math)
        try:
            img = plan.migrate(self.hdr, self.traces)
            V, G = plan.semblance(img, grad=grad)
            if not grad:
                return V, None, None
            g = plan.velocity_grad(self.hdr, G, self.traces).cpu().numpy()
            plan.sync()
            self.evaluations += 1
            return V, float(g[0]), float(g[1])
        finally:
            plan.close()

    def run(self, v0: float, k: float, n_iter: int = 30, scale=(100.0, 0.1), tol: float = 1e-12):
        """Minimises V from (v0, k): BFGS on (v0 / scale[0], k / scale[1]).  Returns a dict with
        the final model, V and the history of (v0, k, V)."""
        sc = np.asarray(scale, dtype=np.float64)
        th = np.array([v0, k], dtype=np.float64)
        V, g0, g1 = self.objective(*th)
        g = np.array([g0, g1]) * sc
        Hinv = np.eye(2)
        hist = [(float(th[0]), float(th[1]), V)]
        for _ in range(n_iter):
            p = -Hinv @ g
            a = 1.0
            while True:   # Armijo backtracking
                tn = th + a * p * sc
                Vn, h0, h1 = self.objective(*tn)
                if Vn <= V + 1e-4 * a * float(g @ p) or a < 1e-3:
                    break
                a *= 0.5
            gn = np.array([h0, h1]) * sc
            step, y = a * p, gn - g
            sy = float(step @ y)
            if sy > 1e-300:   # BFGS update of the inverse Hessian
                r = 1.0 / sy
                eye = np.eye(2)
                Hinv = (eye - r * np.outer(step, y)) @ Hinv @ (eye - r * np.outer(y, step)) + r * np.outer(step, step)
            done = abs(V - Vn) <= tol * max(abs(V), 1e-300)
            th, V, g = tn, Vn, gn
            hist.append((float(th[0]), float(th[1]), V))
            if done:
                break
        return {"v0": float(th[0]), "k": float(th[1]), "V": V, "history": hist,
                "evaluations": self.evaluations}
