"""Lower-level functional, its derivatives and the adjoint Jacobian J (FP64).

Phi(x, theta) = ||A x - y||^2 + R(x, theta) + (l2_eps / 2) ||x||^2
  eq. (1.1) data term (squared, unhalved) plus the eps-term of eq. (5.1).

FoE (eq. (5.1)):  R = sum_j exp(alpha_j) sum_p phi((K_j x)[p]),
  theta = [alpha_1, taps_1, ..., alpha_N, taps_N]   (Section 5, below eq. (5.1)).
TV:               R = exp(theta_0) sum_p sqrt(|(D x)_p|^2 + eps^2).

Hessian H = D^2_xx Phi (eq. (2.6)), adjoint Jacobian J = -(D^2_{theta x} Phi)^T
(Section 3.2), so the hypergradient of eq. (2.7) is J w with H w = grad ell.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops


def phi_fns(kind: str, eps: float):
    """Return (phi, phi', phi'') for the elementwise penalty."""
    if kind == "charbonnier":
        def f(s):
            return np.sqrt(s * s + eps * eps)

        def df(s):
            return s / np.sqrt(s * s + eps * eps)

        def d2f(s):
            return eps * eps / (s * s + eps * eps) ** 1.5
    elif kind == "sq":
        def f(s):
            return s * s

        def df(s):
            return 2.0 * s

        def d2f(s):
            return 2.0 * np.ones_like(s)
    elif kind == "log1p":
        def f(s):
            return np.log1p(s * s)

        def df(s):
            return 2.0 * s / (1.0 + s * s)

        def d2f(s):
            return 2.0 * (1.0 - s * s) / (1.0 + s * s) ** 2
    else:
        raise ValueError(kind)
    return f, df, d2f


class LowerLevel:
    def __init__(self, y: np.ndarray, G: np.ndarray, reg: str, n_filters: int = 0,
                 filter_size: int = 0, phi: str = "charbonnier", phi_eps: float = 0.01,
                 l2_eps: float = 1e-6, mask: np.ndarray = None):
        """G: blur kernel of A; or mask (0/1 per pixel): inpainting, A = diag(mask) (Section 5.1)."""
        self.y = np.asarray(y, dtype=np.float64)
        self.h, self.w = self.y.shape
        self.n = self.h * self.w
        self.G = G
        self.mask = None if mask is None else (np.asarray(mask) != 0).astype(np.float64)
        self.reg = reg
        self.N = n_filters
        self.f = filter_size
        self.phi_kind = phi
        self.eps = phi_eps
        self.l2 = l2_eps
        self.phi, self.dphi, self.d2phi = phi_fns(phi, phi_eps)

    @property
    def p(self) -> int:
        return 1 if self.reg == "tv" else self.N * (self.f * self.f + 1)

    # theta layout (Section 5): per filter one log-weight then its taps
    def split(self, theta):
        T = self.f * self.f
        alphas = np.array([theta[j * (T + 1)] for j in range(self.N)])
        ks = [np.asarray(theta[j * (T + 1) + 1: (j + 1) * (T + 1)]).reshape(self.f, self.f)
              for j in range(self.N)]
        return alphas, ks

    def A(self, x):
        if self.mask is not None:
            return self.mask * x
        return ops.blur(x, self.G)

    def At(self, u):
        if self.mask is not None:
            return self.mask * u
        return ops.blur_adjoint(u, self.G)

    # ---- value, gradient, Hessian action ------------------------------------------------
    def value(self, x, theta) -> float:
        r = self.A(x) - self.y
        v = float(np.sum(r * r)) + 0.5 * self.l2 * float(np.sum(x * x))
        if self.reg == "tv":
            a = ops.grad_fwd(x)
            v += np.exp(theta[0]) * float(np.sum(np.sqrt(a[0] ** 2 + a[1] ** 2 + self.eps ** 2)))
        else:
            alphas, ks = self.split(theta)
            for al, k in zip(alphas, ks):
                v += np.exp(al) * float(np.sum(self.phi(ops.correlate(x, k))))
        return v

    def grad(self, x, theta):
        g = 2.0 * self.At(self.A(x) - self.y) + self.l2 * x
        if self.reg == "tv":
            a = ops.grad_fwd(x)
            s = np.sqrt(a[0] ** 2 + a[1] ** 2 + self.eps ** 2)
            g = g + np.exp(theta[0]) * ops.grad_adj(a / s)
        else:
            alphas, ks = self.split(theta)
            for al, k in zip(alphas, ks):
                g = g + np.exp(al) * ops.correlate_adjoint(self.dphi(ops.correlate(x, k)), k)
        return g

    def hvp(self, x, theta, v):
        """H v = 2 A^T A v + l2 v + D^2_xx R(x, theta) v."""
        hv = 2.0 * self.At(self.A(v)) + self.l2 * v
        if self.reg == "tv":
            a = ops.grad_fwd(x)
            s = np.sqrt(a[0] ** 2 + a[1] ** 2 + self.eps ** 2)
            dv = ops.grad_fwd(v)
            # B_p = (I - a a^T / s^2) / s applied to (D v)_p
            adv = (a[0] * dv[0] + a[1] * dv[1]) / (s * s)
            bd = np.stack([(dv[0] - a[0] * adv) / s, (dv[1] - a[1] * adv) / s])
            hv = hv + np.exp(theta[0]) * ops.grad_adj(bd)
        else:
            alphas, ks = self.split(theta)
            for al, k in zip(alphas, ks):
                u = ops.correlate(x, k)
                hv = hv + np.exp(al) * ops.correlate_adjoint(self.d2phi(u) * ops.correlate(v, k), k)
        return hv

    # ---- adjoint Jacobian --------------------------------------------------------------
    def Jw(self, x, theta, w) -> np.ndarray:
        """J w = -d/dtheta <grad_x Phi(x, theta), w> with w held fixed (eq. (2.7))."""
        if self.reg == "tv":
            a = ops.grad_fwd(x)
            s = np.sqrt(a[0] ** 2 + a[1] ** 2 + self.eps ** 2)
            dw = ops.grad_fwd(w)
            return np.array([-np.exp(theta[0]) * float(np.sum((a[0] * dw[0] + a[1] * dw[1]) / s))])
        alphas, ks = self.split(theta)
        r = self.f // 2
        out = np.zeros(self.p)
        T = self.f * self.f
        for j, (al, k) in enumerate(zip(alphas, ks)):
            u = ops.correlate(x, k)
            kw = ops.correlate(w, k)
            e = self.dphi(u)
            d = self.d2phi(u) * kw
            base = j * (T + 1)
            out[base] = -np.exp(al) * float(np.sum(e * kw))
            for a_ in range(-r, r + 1):
                for b_ in range(-r, r + 1):
                    t = (r + a_) * self.f + (r + b_)
                    out[base + 1 + t] = -np.exp(al) * float(
                        np.sum(e * ops.shift(w, a_, b_) + d * ops.shift(x, a_, b_)))
        return out

    # ---- dense assembly (tiny images only) ---------------------------------------------
    def dense_A(self):
        if self.mask is not None:
            return np.diag(self.mask.reshape(-1))
        return ops.dense_correlation(self.G, self.h, self.w)

    def dense_hessian(self, x, theta) -> np.ndarray:
        A = self.dense_A()
        H = 2.0 * A.T @ A + self.l2 * np.eye(self.n)
        xv = x.reshape(-1)
        if self.reg == "tv":
            D = ops.dense_grad(self.h, self.w)
            a = D @ xv
            n = self.n
            a0, a1 = a[:n], a[n:]
            s = np.sqrt(a0 ** 2 + a1 ** 2 + self.eps ** 2)
            B = np.zeros((2 * n, 2 * n))
            idx = np.arange(n)
            B[idx, idx] = (1.0 - a0 * a0 / s ** 2) / s
            B[idx, n + idx] = (-a0 * a1 / s ** 2) / s
            B[n + idx, idx] = (-a0 * a1 / s ** 2) / s
            B[n + idx, n + idx] = (1.0 - a1 * a1 / s ** 2) / s
            H += np.exp(theta[0]) * D.T @ B @ D
        else:
            alphas, ks = self.split(theta)
            for al, k in zip(alphas, ks):
                K = ops.dense_correlation(k, self.h, self.w)
                u = K @ xv
                H += np.exp(al) * K.T @ np.diag(self.d2phi(u)) @ K
        return H

    def dense_J(self, x, theta) -> np.ndarray:
        """J = -(D^2_{theta x} Phi)^T as a dense p x n matrix, row by row from dense factors."""
        xv = x.reshape(-1)
        n = self.n
        if self.reg == "tv":
            D = ops.dense_grad(self.h, self.w)
            a = D @ xv
            s = np.sqrt(a[:n] ** 2 + a[n:] ** 2 + self.eps ** 2)
            return -np.exp(theta[0]) * (D.T @ (a / np.concatenate([s, s])))[None, :]
        alphas, ks = self.split(theta)
        T = self.f * self.f
        r = self.f // 2
        J = np.zeros((self.p, n))
        for j, (al, k) in enumerate(zip(alphas, ks)):
            K = ops.dense_correlation(k, self.h, self.w)
            u = K @ xv
            e = self.dphi(u)
            dd = self.d2phi(u)
            base = j * (T + 1)
            # d/d alpha of exp(alpha) K^T phi'(K x)
            J[base] = -np.exp(al) * (K.T @ e)
            for a_ in range(-r, r + 1):
                for b_ in range(-r, r + 1):
                    t = (r + a_) * self.f + (r + b_)
                    S = ops.dense_shift(a_, b_, self.h, self.w)
                    # d/dk[o] of K^T phi'(K x) = S_o^T phi'(u) + K^T diag(phi''(u)) S_o x
                    J[base + 1 + t] = -np.exp(al) * (S.T @ e + K.T @ (dd * (S @ xv)))
        return J
