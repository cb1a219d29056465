"""Krylov solvers for the Hessian system H w = g (FP64).

cg      textbook conjugate gradient (Section 2.1 cites it as the standard choice).
rcg     recycled (augmented) CG over a recycle space U with C = H U, C^T C = I
        (Section 2.2.2).  The paper lists only RMINRES (Algorithm 3); rcg applies the
        same augmentation to CG: the initial projection of Algorithm 3 (w0 += U C^T r0,
        r0 -= C C^T r0), then CG on P H P with P = I - C C^T, whose iterates keep
        C^T r = 0, and the recycle-space coefficients z collected along the way so
        that g - H (w + U z) = r holds exactly.
minres  MINRES via the Lanczos relation (2.9)-(2.10) and Givens QR.
rminres Algorithm 3 with the explicit residual of Appendix A.  Reading adopted for
        the garbled update: the recycle part enters the solution with a minus sign,
        w_k = w_{k-1} + c_k zeta_{k-1} (v~_k - b~_k), which is what eq. (2.13)
        (z_k = C^T r0 - C^T H V_k y_k) and the residual recurrence of Appendix A require.

Stopping rules (Section 4): "resid" stops when ||r_k|| < tol; "nsc" stops when the
hypergradient-error estimate ||Z^T r_k|| < tol, Z = W~ V~_H diag(mu) (eq. (4.2)).
The stored Krylov basis V is the list of normalised residuals r_0..r_{k-1}.
"""
from __future__ import annotations

import numpy as np


def cg(apply_H, g, w0, tol, maxit):
    w = w0.copy()
    r = g - apply_H(w)
    p = r.copy()
    rho = float(r @ r)
    it = 0
    while np.sqrt(rho) >= tol and it < maxit:
        q = apply_H(p)
        alpha = rho / float(p @ q)
        w += alpha * p
        r -= alpha * q
        rho_new = float(r @ r)
        p = r + (rho_new / rho) * p
        rho = rho_new
        it += 1
    return w, it, np.sqrt(rho)


def rcg(apply_H, g, w0, U=None, C=None, tol=1e-8, maxit=1000, stop="resid", Z=None,
        store_basis=True, kmax_store=None):
    """Recycled CG; with U = None it is textbook CG that also records its basis.

    Returns dict(w, iters, resid, nsc, V, converged).
    """
    n = g.shape[0]
    w = w0.copy()
    r = g - apply_H(w)
    if U is not None and U.shape[1] > 0:
        c0 = C.T @ r
        w += U @ c0
        r -= C @ c0
        s = U.shape[1]
    else:
        U = np.zeros((n, 0))
        C = np.zeros((n, 0))
        s = 0
    use_nsc = stop == "nsc" and Z is not None and Z.shape[1] > 0

    def measure(rv):
        return float(np.linalg.norm(Z.T @ rv)) if use_nsc else float(np.linalg.norm(rv))

    p = r.copy()
    rho = float(r @ r)
    z = np.zeros(s)
    basis = []
    it = 0
    est = measure(r)
    while est >= tol and it < maxit:
        if store_basis:
            basis.append(r / np.sqrt(rho))
        q = apply_H(p)
        c = C.T @ q
        alpha = rho / float(p @ q)
        w += alpha * p
        z -= alpha * c
        r -= alpha * (q - C @ c)
        rho_new = float(r @ r)
        p = r + (rho_new / rho) * p
        rho = rho_new
        it += 1
        est = measure(r)
    if s:
        w += U @ z
    if kmax_store is not None and len(basis) > kmax_store:
        basis = basis[-kmax_store:]
    V = np.array(basis).T if basis else np.zeros((n, 0))
    return dict(w=w, iters=it, resid=np.sqrt(rho), nsc=(measure(r) if use_nsc else None),
                V=V, converged=est < tol, r=r)


def minres(apply_H, g, w0, tol, maxit):
    return rminres(apply_H, g, w0, None, None, tol, maxit)


def rminres(apply_H, g, w0, U, C, tol=1e-8, maxit=1000, stop="resid", Z=None):
    """Algorithm 3 (RMINRES) with the explicit residual recurrence of Appendix A."""
    n = g.shape[0]
    if U is None:
        U = np.zeros((n, 0))
        C = np.zeros((n, 0))
    w = w0.copy()
    r = g - apply_H(w)
    c0 = C.T @ r
    w = w + U @ c0
    r = r - C @ c0
    beta = np.linalg.norm(r)
    res = r.copy()                       # explicit residual (Appendix A)
    v_prev = np.zeros(n)
    v = r / beta if beta > 0 else r.copy()
    zeta = beta
    vt_m2 = np.zeros(n)
    vt_m1 = np.zeros(n)
    bt_m2 = np.zeros(n)
    bt_m1 = np.zeros(n)
    Hvt_m2 = np.zeros(n)
    Hvt_m1 = np.zeros(n)
    Hbt_m2 = np.zeros(n)
    Hbt_m1 = np.zeros(n)
    c_m1, s_m1, c_m2, s_m2 = 1.0, 0.0, 0.0, 0.0
    basis = []
    use_nsc = stop == "nsc" and Z is not None and Z.shape[1] > 0

    def measure(rv):
        return float(np.linalg.norm(Z.T @ rv)) if use_nsc else abs(zeta)

    it = 0
    while it < maxit and measure(res) >= tol and beta > 0:
        basis.append(v.copy())
        Hv = apply_H(v)
        cHv = C.T @ Hv
        b = U @ cHv
        CcHv = C @ cHv
        vn = Hv - CcHv
        alpha = float(v @ vn)
        vn = vn - alpha * v - beta * v_prev
        beta_next = np.linalg.norm(vn)
        gamma = s_m2 * beta
        delta = c_m1 * c_m2 * beta + s_m1 * alpha
        eps = -s_m1 * c_m2 * beta + c_m1 * alpha
        eps_t = np.hypot(eps, beta_next)
        s_k = beta_next / eps_t
        c_k = eps / eps_t
        zeta_prev = zeta
        zeta = -s_k * zeta_prev
        vt = (v - gamma * vt_m2 - delta * vt_m1) / eps_t
        bt = (b - gamma * bt_m2 - delta * bt_m1) / eps_t
        Hvt = (Hv - gamma * Hvt_m2 - delta * Hvt_m1) / eps_t
        Hbt = (CcHv - gamma * Hbt_m2 - delta * Hbt_m1) / eps_t
        w = w + c_k * zeta_prev * (vt - bt)
        res = res - c_k * zeta_prev * (Hvt - Hbt)
        vt_m2, vt_m1 = vt_m1, vt
        bt_m2, bt_m1 = bt_m1, bt
        Hvt_m2, Hvt_m1 = Hvt_m1, Hvt
        Hbt_m2, Hbt_m1 = Hbt_m1, Hbt
        c_m2, s_m2, c_m1, s_m1 = c_m1, s_m1, c_k, s_k
        v_prev = v
        v = vn / beta_next if beta_next > 0 else vn
        beta = beta_next
        it += 1
    V = np.array(basis).T if basis else np.zeros((n, 0))
    return dict(w=w, iters=it, resid=abs(zeta), r=res, V=V,
                nsc=(float(np.linalg.norm(Z.T @ res)) if use_nsc else None))
