"""Recycle-space selection (Section 3) and the hypergradient-error estimate (Section 4), FP64.

All routines take W~, an orthonormal basis of range(W), W = [U^(i-1), V^(i-1)]
(reading adopted: W is orthonormalised first, which makes W = I the exact
full-space limit the paper states after eq. (3.1) and after eq. (3.4)).

ritz             eq. (3.1): W~^T H W~ = Q Lambda Q^T, Ritz vectors W~ Q (returns Q_sel).
harmonic_ritz    eq. (3.2): (H W~)^T H W~ rho = theta (H W~)^T W~ rho, vectors W~ rho
                 (returns rho_sel).
gsvd_paige_saunders  GSVD of (J~, T) as in Paige-Saunders: QR of [J~; T], SVD of the
                 lower block, column normalisation of the upper block (Theorem 3.1).
gsvd_closed_form J~ T^{-1} = V_J diag(mu) V_H^T (eq. (3.4)), X = T^{-1} V_H D_H,
                 D_H = diag(1 / sqrt(1 + mu^2)), D_J = diag(mu) D_H.
rgsv             Ritz generalized singular vectors, sides R (W~ X), L (W~ V_H),
                 M (the average), sizes S / L / M (Table 1).
qr_normalise     H U~ = C R, U = U~ R^{-1}, so that C = H U and C^T C = I (Section 2.2.2).
refresh          the outer variant (eq. (3.3)): W projected with the current Hessian H^(i).
refresh_inner    the inner variant (eq. (3.4)): W projected with the previous Hessian H^(i-1)
                 (the one the basis V was built with); the selected U~ is then paired with
                 C = H^(i) U (QR-normalised) for the new system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def orth_basis(W: np.ndarray, rtol: float = 1e-10) -> np.ndarray:
    """Orthonormal basis of range(W), dropping directions with sigma < rtol * sigma_max."""
    if W.shape[1] == 0:
        return W
    Q, sv, _ = np.linalg.svd(W, full_matrices=False)
    keep = sv > rtol * sv[0]
    return Q[:, keep]


def _select(order_len: int, s: int, which: str) -> np.ndarray:
    """Indices into ascending-sorted values: smallest, largest or half of each."""
    s = min(s, order_len)
    if which == "S":
        return np.arange(s)
    if which == "L":
        return np.arange(order_len - s, order_len)
    if which == "M":
        lo = s - s // 2
        hi = s // 2
        return np.concatenate([np.arange(lo), np.arange(order_len - hi, order_len)])
    raise ValueError(which)


def ritz(Wt, HWt, s, which="S"):
    T = Wt.T @ HWt
    T = 0.5 * (T + T.T)
    lam, Q = np.linalg.eigh(T)
    idx = _select(len(lam), s, which)
    return Q[:, idx], lam[idx]


def harmonic_ritz(Wt, HWt, s, which="S"):
    a = HWt.T @ HWt
    b = HWt.T @ Wt
    a = 0.5 * (a + a.T)
    b = 0.5 * (b + b.T)
    th, R = sla.eigh(a, b)
    idx = _select(len(th), s, which)
    return R[:, idx], th[idx]


def gsvd_paige_saunders(Jt: np.ndarray, T: np.ndarray):
    """GSVD of the pair (J~ in R^{p x t}, T in R^{t x t}, invertible).

    Returns mu (ascending), X, V_H, V_J (thin), alpha, beta with
    J~ X = V_J diag(alpha), T X = V_H diag(beta), alpha^2 + beta^2 = 1.
    """
    p, t = Jt.shape
    Q, R = np.linalg.qr(np.vstack([Jt, T]))
    Q1, Q2 = Q[:p], Q[p:]
    VH, beta, Zt = np.linalg.svd(Q2)          # Q2 = V_H diag(beta) Z^T, beta descending
    Zm = Zt.T
    Q1Z = Q1 @ Zm
    alpha = np.linalg.norm(Q1Z, axis=0)
    VJ = np.zeros_like(Q1Z)
    nz = alpha > 1e-300
    VJ[:, nz] = Q1Z[:, nz] / alpha[nz]
    X = np.linalg.solve(R, Zm)
    mu = alpha / beta
    order = np.argsort(mu, kind="stable")
    return dict(mu=mu[order], X=X[:, order], VH=VH[:, order], VJ=VJ[:, order],
                alpha=alpha[order], beta=beta[order])


def gsvd_closed_form(Jt: np.ndarray, T: np.ndarray):
    p, t = Jt.shape
    B = np.linalg.solve(T.T, Jt.T).T           # J~ T^{-1}
    VJ, mu, VHt = np.linalg.svd(B, full_matrices=True)
    mu_full = np.zeros(t)
    mu_full[:min(p, t)] = mu[:min(p, t)]
    VH = VHt.T
    DH = 1.0 / np.sqrt(1.0 + mu_full ** 2)
    X = np.linalg.solve(T, VH) * DH[None, :]
    order = np.argsort(mu_full, kind="stable")
    return dict(mu=mu_full[order], X=X[:, order], VH=VH[:, order],
                alpha=(mu_full * DH)[order], beta=DH[order])


def rgsv(Wt, HWt, JWt, s, which="L", side="R", method="closed"):
    """Ritz generalized singular vectors of (J W~, W~^T H W~) and the NSC operator Z.

    Returns (Y, Z, mu_selected) with U~ = W~ Y.  Z = W~ V_H[:, sel] diag(mu_sel)
    so that ||Z^T r|| is the estimate of eq. (4.2).
    """
    T = Wt.T @ HWt
    T = 0.5 * (T + T.T)
    dec = gsvd_closed_form(JWt, T) if method == "closed" else gsvd_paige_saunders(JWt, T)
    idx = _select(len(dec["mu"]), s, which)
    if side == "R":
        Y = dec["X"][:, idx]
    elif side == "L":
        Y = dec["VH"][:, idx]
    elif side == "M":
        Y = 0.5 * (dec["VH"][:, idx] + dec["X"][:, idx])
    else:
        raise ValueError(side)
    Z = Wt @ (dec["VH"][:, idx] * dec["mu"][idx][None, :])
    return Y, Z, dec["mu"][idx]


def qr_normalise(Ut: np.ndarray, HUt: np.ndarray):
    """H U~ = C R (reduced QR), U = U~ R^{-1}: C = H U, C^T C = I, range(U) = range(U~)."""
    C, R = np.linalg.qr(HUt)
    U = sla.solve_triangular(R, Ut.T, trans="T", lower=False).T
    return U, C


def nsc_estimate(Z: np.ndarray, r: np.ndarray) -> float:
    """||D~_J D~_H^{-1} V~_H^T W^T r|| = ||Z^T r|| (eq. (4.2))."""
    return float(np.linalg.norm(Z.T @ r))


def refresh(U_prev, V_prev, apply_H, apply_J, s, kind="rgsv", which="L", side="R",
            rtol=1e-10):
    """Outer recycle refresh (Section 3.1, eq. (3.3)): W = [U^(i-1), V^(i-1)], projected
    with the current H^(i) (and J^(i) for Ritz generalized singular vectors).

    apply_H(v) and apply_J(v) act on one n-vector.  Returns (U, C, Z, values) with
    C = H U, C^T C = I; Z is None unless kind == "rgsv".
    """
    W = np.hstack([U_prev, V_prev])
    Wt = orth_basis(W, rtol)
    HWt = np.stack([apply_H(Wt[:, j]) for j in range(Wt.shape[1])], axis=1)
    Z = None
    if kind == "ritz":
        Y, vals = ritz(Wt, HWt, s, which)
    elif kind == "hritz":
        Y, vals = harmonic_ritz(Wt, HWt, s, which)
    elif kind == "rgsv":
        JWt = np.stack([apply_J(Wt[:, j]) for j in range(Wt.shape[1])], axis=1)
        Y, Z, vals = rgsv(Wt, HWt, JWt, s, which, side)
    else:
        raise ValueError(kind)
    U, C = qr_normalise(Wt @ Y, HWt @ Y)
    return U, C, Z, vals


def refresh_inner(U_prev, V_prev, apply_H_old, apply_H_new, apply_J, s, kind="ritz", which="S", side="R",
                  rtol=1e-10):
    """Inner recycle refresh (Section 3.1, eq. (3.4)): W = [U^(i-1), V^(i-1)], the projected
    problem built with H^(i-1) (J at the current point for Ritz generalized singular vectors);
    then C = H^(i) U~ R^{-1} by QR (Section 2.2.2), so the new system's C = H U, C^T C = I.
    Returns (U, C, Z, values) as refresh()."""
    W = np.hstack([U_prev, V_prev])
    Wt = orth_basis(W, rtol)
    HWt = np.stack([apply_H_old(Wt[:, j]) for j in range(Wt.shape[1])], axis=1)
    Z = None
    if kind == "ritz":
        Y, vals = ritz(Wt, HWt, s, which)
    elif kind == "hritz":
        Y, vals = harmonic_ritz(Wt, HWt, s, which)
    elif kind == "rgsv":
        JWt = np.stack([apply_J(Wt[:, j]) for j in range(Wt.shape[1])], axis=1)
        Y, Z, vals = rgsv(Wt, HWt, JWt, s, which, side)
    else:
        raise ValueError(kind)
    Ut = Wt @ Y
    HUt = np.stack([apply_H_new(Ut[:, j]) for j in range(Ut.shape[1])], axis=1)
    U, C = qr_normalise(Ut, HUt)
    return U, C, Z, vals

