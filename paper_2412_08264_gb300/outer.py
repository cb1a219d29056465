"""Outer (upper-level) drivers over the C ABI: one hypergradient per pair per step.

Engine: the hot path for one batch (eq. (5.2)) — warm-started lower solve, recycle refresh,
warm-started recycled-CG Hessian solve, J w — with the recycle state, x^ and w kept between calls
(the sequence of Hessian systems, eq. (2.8), is what recycling exploits).

gradient_descent  Algorithms 1 and 2 (step theta - beta rho^{j-1} d, Armijo test
                  L(theta_j) < L(theta) - eta beta rho^{j-1} ||d||^2, warm-started trial solves,
                  next initial step 2 beta rho^{j-1}).
adam              Adam with a fixed step length (Section 5.2).
The few theta-sized (p values) updates run on the host in FP64; every per-pixel operation runs in
libbl's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import api
from .strategy import Strategy, parse


@dataclass
class StepInfo:
    loss: float
    hg_norm: float
    krylov_iters: List[int]
    lower_iters: List[int]
    extra: dict = field(default_factory=dict)


class Engine:
    def __init__(self, problem: api.Problem, strategy="RGen-L(R)", s: int = 16, rtol: float = 1e-4,
                 lower_gtol: float = 1e-5, lower_max_iters: int = 5000, maxit: int = 5000,
                 nsc_tol: Optional[float] = None, lower_relative: bool = True, method: str = "cg",
                 refresh: str = "outer"):
        self.P = problem
        self.method = method            # "cg" (SPD Hessians) or "minres" (Algorithm 3, indefinite)
        self.refresh = refresh          # "outer" (eq. (3.3)) or "inner" (eq. (3.4), CG only)
        self.strategy: Strategy = parse(strategy) if isinstance(strategy, str) else strategy
        self.s = s
        self.rtol = rtol
        self.nsc_tol = nsc_tol
        self.lower_gtol = lower_gtol
        self.lower_max_iters = lower_max_iters
        self.lower_relative = lower_relative
        self.maxit = maxit
        self.xhat = problem.zeros()
        self.w = problem.zeros()
        self.n_systems = 0
        self.hg_prev = None

    # ---- pieces ----------------------------------------------------------------------
    def lower(self, theta: torch.Tensor, x0: Optional[torch.Tensor] = None):
        x = (self.xhat if x0 is None else x0).clone()
        info = self.P.lower_solve(theta, x, gtol=self.lower_gtol, relative=self.lower_relative,
                                  max_iters=self.lower_max_iters, allow_noconv=True)
        return x, info

    def hypergrad_at_point(self, g: Optional[torch.Tensor] = None, per_pair: bool = False):
        """Refresh + recycled solve + J w at the point set by the last lower solve / set_point."""
        st = self.strategy
        if st.recycles and self.n_systems > 0:
            self.P.ritz_update(st, self.s, variant=self.refresh)
        nsc = st.nsc and self.nsc_tol is not None
        tol = self.nsc_tol if nsc else self.rtol
        scale = None if (not nsc or self.hg_prev is None) else [self.hg_prev] * self.P.K
        info = self.P.hessian_solve(self.w, g=g, recycle=st.recycles, nsc=nsc, tol=tol, relative=True,
                                    maxit=self.maxit,
                                    store_basis=(("lanczos" if self.refresh == "inner" else True) if st.recycles
                                                 else False),
                                    warm_start=True, nsc_scale=scale,
                                    allow_noconv=True, method=self.method)
        self.n_systems += 1
        mean, per, loss = self.P.hypergrad(self.w, per_pair=True, loss=True)
        self.hg_prev = float(mean.norm())
        return (mean, per, loss, info) if per_pair else (mean, loss, info)

    def loss_and_hypergrad(self, theta: torch.Tensor):
        x, linfo = self.lower(theta)
        self.xhat = x
        mean, loss, kinfo = self.hypergrad_at_point()
        return loss, mean, StepInfo(loss, float(mean.norm()), [i["iters"] for i in kinfo],
                                    [i["iters"] for i in linfo])

    # ---- checkpoint (recycle space, point, solution) ----------------------------------
    def state_dict(self) -> dict:
        return {"recycle": [self.P.recycle_export(k) for k in range(self.P.K)],
                "xhat": self.xhat.detach().cpu(), "w": self.w.detach().cpu(), "n_systems": self.n_systems,
                "hg_prev": self.hg_prev}

    def load_state_dict(self, sd: dict):
        for k, blob in enumerate(sd["recycle"]):
            self.P.recycle_import(k, blob)
        self.xhat = sd["xhat"].to(self.P.device)
        self.w = sd["w"].to(self.P.device)
        self.n_systems = sd["n_systems"]
        self.hg_prev = sd["hg_prev"]


def gradient_descent(engine: Engine, theta0: np.ndarray, steps: int, beta0: float = 1.0, rho: float = 0.5,
                     eta: float = 1e-4, max_backtrack: int = 30):
    """Algorithms 1 and 2 on the GPU engine.  Returns (theta, history)."""
    dev = engine.P.device
    theta = np.array(theta0, dtype=np.float64)
    th_d = torch.tensor(theta, dtype=torch.float64, device=dev)
    x, _ = engine.lower(th_d)          # also sets the point (theta, x^) in the library
    engine.xhat = x
    beta = beta0
    hist = []
    for _ in range(steps):
        mean, c1, kinfo = engine.hypergrad_at_point()
        d = mean.cpu().numpy()
        dd = float(d @ d)
        xt = engine.xhat
        for j in range(1, max_backtrack + 1):
            step = beta * rho ** (j - 1)
            th_j = theta - step * d
            th_jd = torch.tensor(th_j, dtype=torch.float64, device=dev)
            xt, _ = engine.lower(th_jd, xt)
            _, c0 = engine.P.hypergrad(engine.w, loss=True)
            if c0 < c1 - eta * step * dd:
                break
        beta = 2.0 * step
        theta = th_j
        engine.xhat = xt
        hist.append(StepInfo(c0, np.sqrt(dd), [i["iters"] for i in kinfo], [], {"step": step}))
    return theta, hist


def adam(engine: Engine, theta0: np.ndarray, steps: int, lr: float = 1e-2, b1: float = 0.9, b2: float = 0.999,
         eps: float = 1e-8, checkpoint_every: int = 0, checkpoints: Optional[list] = None):
    """Adam with a fixed step length (Section 5.2) on the GPU engine."""
    dev = engine.P.device
    theta = np.array(theta0, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    hist = []
    for t in range(1, steps + 1):
        loss, mean, info = engine.loss_and_hypergrad(torch.tensor(theta, dtype=torch.float64, device=dev))
        g = mean.cpu().numpy()
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        theta = theta - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        hist.append(info)
        if checkpoint_every and checkpoints is not None and t % checkpoint_every == 0:
            checkpoints.append((t, theta.copy(), engine.state_dict()))
    return theta, hist
