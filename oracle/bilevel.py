"""Bilevel problem over K training pairs (eq. (5.2)) and its outer solvers, FP64.

Upper loss (reading adopted for eqs. (1.2) / (5.2)): L = (1/K) sum_k 1/2 ||x^_k - x*_k||^2,
so grad ell_k = x^_k - x*_k and the hypergradient is (1/K) sum_k J_k w_k with
H_k w_k = x^_k - x*_k (eqs. (2.6), (2.7)).

gradient_descent  Algorithms 1 and 2: step theta - beta rho^{j-1} d, Armijo test
                  L(theta_j) < L(theta) - eta beta rho^{j-1} ||d||^2, warm-started lower
                  solves, next initial step 2 beta rho^{j-1}.
adam              Adam with a fixed step length (Section 5.2).
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .functional import LowerLevel
from .krylov import cg
from .lbfgs import lbfgs


class BilevelProblem:
    def __init__(self, wl):
        """wl: a paper_2412_08264_gb300.synth.Workload (seeded images, noise, theta0)."""
        self.wl = wl
        self.K = len(wl.pairs)
        self.lowers = []
        self.ys = []
        masks = (list(getattr(wl, "masks", None) or []) + [None] * self.K)[:self.K]
        for spec, xs, nz, m in zip(wl.pairs, wl.x_star, wl.noise, masks):
            if m is not None:
                # inpainting (Section 5.1): only the measured pixels carry data
                G = None
                y = (m != 0) * (xs + nz)
            else:
                G = ops.gaussian_kernel(spec.blur_sigma, spec.blur_radius)
                y = ops.blur(xs, G) + nz
            self.ys.append(y)
            self.lowers.append(LowerLevel(y, G, wl.reg, wl.n_filters, wl.filter_size,
                                          wl.phi, wl.phi_eps, wl.l2_eps, mask=m))
        self.x_star = wl.x_star

    @property
    def p(self):
        return self.lowers[0].p

    def solve_lower(self, theta, x0s=None, gtol=1e-8, m=10):
        xs, infos = [], []
        for k, ll in enumerate(self.lowers):
            x0 = np.zeros((ll.h, ll.w)) if x0s is None else x0s[k]
            x, info = lbfgs(lambda v: ll.value(v.reshape(ll.h, ll.w), theta),
                            lambda v: ll.grad(v.reshape(ll.h, ll.w), theta).reshape(-1),
                            x0.reshape(-1), gtol, m=m)
            xs.append(x.reshape(ll.h, ll.w))
            infos.append(info)
        return xs, infos

    def loss(self, xhats):
        return float(np.mean([0.5 * np.sum((x - xs) ** 2) for x, xs in zip(xhats, self.x_star)]))

    def rhs(self, k, xhat):
        return (xhat - self.x_star[k]).reshape(-1)

    def apply_H(self, k, xhat, theta):
        ll = self.lowers[k]
        return lambda v: ll.hvp(xhat, theta, v.reshape(ll.h, ll.w)).reshape(-1)

    def Jw(self, k, xhat, theta, w):
        ll = self.lowers[k]
        return ll.Jw(xhat, theta, w.reshape(ll.h, ll.w))

    def reference_w(self, k, xhat, theta, rtol=1e-13, maxit=100000):
        """High-accuracy w* (Section 5: residual tolerance 1e-13): dense Cholesky when n is small."""
        ll = self.lowers[k]
        g = self.rhs(k, xhat)
        if ll.n <= 1600:
            import scipy.linalg as sla
            H = ll.dense_hessian(xhat, theta)
            return sla.cho_solve(sla.cho_factor(H), g)
        w, _, _ = cg(self.apply_H(k, xhat, theta), g, np.zeros_like(g),
                     rtol * np.linalg.norm(g), maxit)
        return w

    def hypergradient(self, theta, xhats, ws):
        return np.mean([self.Jw(k, xhats[k], theta, ws[k]) for k in range(self.K)], axis=0)


def gradient_descent(prob: BilevelProblem, theta0, n_steps, solve_hessian, beta0=1.0, rho=0.5,
                     eta=1e-4, gtol_lower=1e-8, max_backtrack=30, log=None):
    """Algorithm 2 with Algorithm 1; solve_hessian(k, xhat, theta, g) -> w."""
    theta = np.array(theta0, dtype=np.float64)
    xhats, _ = prob.solve_lower(theta, gtol=gtol_lower)
    c1 = prob.loss(xhats)
    beta = beta0
    thetas = [theta.copy()]
    for i in range(n_steps):
        ws = [solve_hessian(k, xhats[k], theta, prob.rhs(k, xhats[k])) for k in range(prob.K)]
        d = prob.hypergradient(theta, xhats, ws)
        dd = float(d @ d)
        xt = xhats
        for j in range(1, max_backtrack + 1):
            step = beta * rho ** (j - 1)
            th_j = theta - step * d
            xt, _ = prob.solve_lower(th_j, xt, gtol=gtol_lower)
            c0 = prob.loss(xt)
            if c0 < c1 - eta * step * dd:
                break
        beta = 2.0 * step
        theta, xhats, c1 = th_j, xt, c0
        thetas.append(theta.copy())
        if log is not None:
            log.append(dict(step=i, loss=c1, hg_norm=np.sqrt(dd), step_len=step))
    return theta, xhats, thetas


class Adam:
    def __init__(self, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = None
        self.v = None
        self.t = 0

    def step(self, theta, g):
        if self.m is None:
            self.m = np.zeros_like(theta)
            self.v = np.zeros_like(theta)
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
