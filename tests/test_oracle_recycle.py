"""Pins for recycle-space selection (Section 3) and the error estimate (Section 4).

W = I limits (exact eigendecomposition, exact GSVD), J W = I (reciprocal Ritz
values), alpha^2 + beta^2 = 1 and orderings (Theorem 3.1), two independent
GSVD constructions, the QR normalisation, and the equality case of eq. (4.2).
"""
import numpy as np
import pytest

from oracle import recycle as rc


def spd(rng, n, cond=1e3):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(cond), n)
    return (Q * lam) @ Q.T


def test_qr_normalise(rng):
    n, s = 30, 5
    H = spd(rng, n)
    Ut = rng.standard_normal((n, s))
    U, C = rc.qr_normalise(Ut, H @ Ut)
    np.testing.assert_allclose(C.T @ C, np.eye(s), atol=1e-12)
    np.testing.assert_allclose(H @ U, C, atol=1e-10)
    # range(U) = range(U~): projecting U~ on range(U) reproduces it
    Q, _ = np.linalg.qr(U)
    np.testing.assert_allclose(Q @ (Q.T @ Ut), Ut, atol=1e-10)


def test_ritz_full_space_is_eigendecomposition(rng):
    n = 20
    H = spd(rng, n, 50)
    Wt = np.eye(n)
    Q, lam = rc.ritz(Wt, H, 5, "S")
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(H)[:5], rtol=1e-12)
    np.testing.assert_allclose(H @ Q, Q * lam, atol=1e-10)
    _, laml = rc.ritz(Wt, H, 3, "L")
    np.testing.assert_allclose(laml, np.linalg.eigvalsh(H)[-3:], rtol=1e-12)
    _, lamm = rc.ritz(Wt, H, 4, "M")
    ev = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(lamm, np.concatenate([ev[:2], ev[-2:]]), rtol=1e-12)


def test_ritz_values_interlace(rng):
    """Ritz values on a subspace lie inside the spectrum (Cauchy interlacing)."""
    n, t = 40, 8
    H = spd(rng, n, 1e3)
    Wt = rc.orth_basis(rng.standard_normal((n, t)))
    _, lam = rc.ritz(Wt, H @ Wt, t, "S")
    ev = np.linalg.eigvalsh(H)
    assert lam.min() >= ev[0] - 1e-9 and lam.max() <= ev[-1] + 1e-9
    for i in range(t):
        assert ev[i] - 1e-9 <= lam[i] <= ev[n - t + i] + 1e-9


def test_harmonic_ritz_full_space_is_eigendecomposition(rng):
    n = 15
    H = spd(rng, n, 20)
    R, th = rc.harmonic_ritz(np.eye(n), H, 4, "S")
    np.testing.assert_allclose(th, np.linalg.eigvalsh(H)[:4], rtol=1e-10)


@pytest.mark.parametrize("p,t", [(12, 6), (6, 6), (3, 7)])
def test_gsvd_constructions_agree(p, t, rng):
    Jt = rng.standard_normal((p, t))
    T = spd(rng, t, 30)
    a = rc.gsvd_paige_saunders(Jt, T)
    b = rc.gsvd_closed_form(Jt, T)
    np.testing.assert_allclose(a["mu"], b["mu"], rtol=1e-9, atol=1e-12)
    # Theorem 3.1: alpha^2 + beta^2 = 1, alpha ascending, beta descending
    np.testing.assert_allclose(a["alpha"] ** 2 + a["beta"] ** 2, 1.0, atol=1e-12)
    np.testing.assert_allclose(b["alpha"] ** 2 + b["beta"] ** 2, 1.0, atol=1e-12)
    assert np.all(np.diff(a["mu"]) >= -1e-12)
    assert np.all(np.diff(a["alpha"]) >= -1e-12) and np.all(np.diff(a["beta"]) <= 1e-12)
    # defining relations T X = V_H D_H for both; J X = V_J D_J for Paige-Saunders
    for d in (a, b):
        np.testing.assert_allclose(T @ d["X"], d["VH"] * d["beta"], atol=1e-9)
        np.testing.assert_allclose(d["VH"].T @ d["VH"], np.eye(t), atol=1e-10)
    np.testing.assert_allclose(Jt @ a["X"], a["VJ"] * a["alpha"], atol=1e-9)
    # X columns agree up to sign where mu is simple and non-zero
    for j in range(t):
        if a["mu"][j] > 1e-8:
            xa, xb = a["X"][:, j], b["X"][:, j]
            assert min(np.linalg.norm(xa - xb), np.linalg.norm(xa + xb)) < 1e-7 * np.linalg.norm(xa)
    if p < t:
        assert np.sum(a["mu"] < 1e-10) == t - p    # reading C11: min(p, t) non-zero values


def test_gsvd_with_identity_J_gives_reciprocal_ritz_values(rng):
    """If J W = I, the Ritz generalized singular values are 1 / Ritz values."""
    t = 7
    T = spd(rng, t, 40)
    d = rc.gsvd_closed_form(np.eye(t), T)
    np.testing.assert_allclose(np.sort(d["mu"]), np.sort(1.0 / np.linalg.eigvalsh(T)), rtol=1e-10)
    d2 = rc.gsvd_paige_saunders(np.eye(t), T)
    np.testing.assert_allclose(np.sort(d2["mu"]), np.sort(1.0 / np.linalg.eigvalsh(T)), rtol=1e-9)


def test_rgsv_full_space_is_gsvd_of_J_H(rng):
    """W = I: the right RGSVs satisfy J X = V_J D_J, H X = V_H D_H with the full J and H."""
    n, p = 10, 14
    H = spd(rng, n, 20)
    J = rng.standard_normal((p, n))
    d = rc.gsvd_paige_saunders(J, H)
    np.testing.assert_allclose(H @ d["X"], d["VH"] * d["beta"], atol=1e-10)
    np.testing.assert_allclose(J @ d["X"], d["VJ"] * d["alpha"], atol=1e-10)
    # and the singular values of J H^{-1} are the generalized singular values
    np.testing.assert_allclose(d["mu"], np.sort(np.linalg.svd(J @ np.linalg.inv(H), compute_uv=False)),
                               rtol=1e-9)


def test_nsc_is_exact_with_full_gsvd(rng):
    """With W square orthogonal and the full GSVD, ||Z^T r|| = ||J H^{-1} r|| (Section 4)."""
    n, p = 12, 16
    H = spd(rng, n, 100)
    J = rng.standard_normal((p, n))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Y, Z, mu = rc.rgsv(Q, H @ Q, J @ Q, n, "L", "R")
    r = rng.standard_normal(n)
    assert abs(rc.nsc_estimate(Z, r) - np.linalg.norm(J @ np.linalg.solve(H, r))) < 1e-9 * np.linalg.norm(r) * 100


def test_refresh_produces_valid_recycle_space(rng):
    n, s = 40, 5
    H = spd(rng, n, 1e3)
    J = rng.standard_normal((9, n))
    Up = rng.standard_normal((n, 4))
    Vp = rc.orth_basis(rng.standard_normal((n, 10)))
    for kind, which in [("ritz", "S"), ("rgsv", "L"), ("hritz", "L")]:
        U, C, Z, vals = rc.refresh(Up, Vp, lambda v: H @ v, lambda v: J @ v, s, kind, which)
        assert U.shape == (n, s)
        np.testing.assert_allclose(H @ U, C, atol=1e-8)
        np.testing.assert_allclose(C.T @ C, np.eye(s), atol=1e-10)
        W = np.hstack([Up, Vp])
        Qw, _ = np.linalg.qr(W)
        np.testing.assert_allclose(Qw @ (Qw.T @ U), U, atol=1e-8 * np.abs(U).max())   # U in range(W)
        if kind == "rgsv":
            assert Z.shape == (n, s) and np.all(np.diff(vals) >= 0)


def test_orth_basis_drops_dependent_columns(rng):
    A = rng.standard_normal((20, 4))
    W = np.hstack([A, A[:, :2] @ rng.standard_normal((2, 3))])
    Wt = rc.orth_basis(W)
    assert Wt.shape == (20, 4)
    np.testing.assert_allclose(Wt.T @ Wt, np.eye(4), atol=1e-12)


def test_refresh_inner_reduces_to_outer_when_the_hessian_is_unchanged(rng):
    """eq. (3.4) with H^(i-1) = H^(i) is eq. (3.3): the same recycle space, C and U."""
    n, s = 40, 5
    H = spd(rng, n, 1e3)
    J = rng.standard_normal((9, n))
    Up = rng.standard_normal((n, 4))
    Vp = rc.orth_basis(rng.standard_normal((n, 10)))
    for kind, which in [("ritz", "S"), ("rgsv", "L"), ("hritz", "L")]:
        U1, C1, Z1, v1 = rc.refresh(Up, Vp, lambda v: H @ v, lambda v: J @ v, s, kind, which)
        U2, C2, Z2, v2 = rc.refresh_inner(Up, Vp, lambda v: H @ v, lambda v: H @ v, lambda v: J @ v, s, kind, which)
        np.testing.assert_allclose(v1, v2, rtol=1e-10)
        np.testing.assert_allclose(C1, C2, atol=1e-9)
        np.testing.assert_allclose(U1, U2, atol=1e-9 * np.abs(U1).max())


def test_refresh_inner_selects_with_the_old_hessian(rng):
    """The inner space is the Ritz space of H^(i-1) on W; its C pairs it with H^(i)."""
    n, s = 40, 5
    Hold = spd(rng, n, 1e3)
    E = rng.standard_normal((n, n))
    Hnew = Hold + 0.05 * (E + E.T)
    Up = rng.standard_normal((n, 4))
    Vp = rc.orth_basis(rng.standard_normal((n, 10)))
    U, C, _, vals = rc.refresh_inner(Up, Vp, lambda v: Hold @ v, lambda v: Hnew @ v, None, s, "ritz", "S")
    Uo, _, _, valso = rc.refresh(Up, Vp, lambda v: Hold @ v, None, s, "ritz", "S")
    np.testing.assert_allclose(vals, valso, rtol=1e-10)
    # same subspace as the outer selection with the old Hessian
    Q1, _ = np.linalg.qr(U)
    Q2, _ = np.linalg.qr(Uo)
    assert np.linalg.svd(Q1.T @ Q2, compute_uv=False).min() > 1 - 1e-10
    np.testing.assert_allclose(Hnew @ U, C, atol=1e-8)
    np.testing.assert_allclose(C.T @ C, np.eye(s), atol=1e-10)
