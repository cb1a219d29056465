"""Pins for the Krylov solvers (Section 2.2, Algorithm 3, Appendix A).

CG against a dense solve; recycled CG with an empty recycle space against
textbook CG; recycled CG against its defining Galerkin conditions (brute force
on a tiny system); RMINRES against the dense least-squares problems (2.11) and
(2.13) it solves.
"""
import numpy as np
import pytest

from oracle.krylov import cg, rcg, rminres, minres
from oracle.recycle import qr_normalise


def spd(rng, n, cond=1e3):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(cond), n)
    return (Q * lam) @ Q.T


def test_cg_matches_dense_solve(rng):
    n = 30
    H = spd(rng, n)
    g = rng.standard_normal(n)
    w, it, res = cg(lambda v: H @ v, g, np.zeros(n), 1e-12, 500)
    np.testing.assert_allclose(w, np.linalg.solve(H, g), rtol=1e-9)
    assert res < 1e-12


def test_cg_terminates_within_n_steps_on_few_eigenvalues(rng):
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat([1.0, 2.0, 5.0, 7.0], 10)   # 4 distinct eigenvalues -> at most 4 steps
    H = (Q * lam) @ Q.T
    g = rng.standard_normal(n)
    w, it, res = cg(lambda v: H @ v, g, np.zeros(n), 1e-10, 100)
    assert it <= 4 + 1


def test_rcg_without_recycling_is_textbook_cg(rng):
    n = 25
    H = spd(rng, n, 1e2)
    g = rng.standard_normal(n)
    w0 = rng.standard_normal(n)
    for k in [1, 3, 7]:
        wa, ita, _ = cg(lambda v: H @ v, g, w0, 0.0, k)
        out = rcg(lambda v: H @ v, g, w0, None, None, tol=0.0, maxit=k)
        assert out["iters"] == ita == k
        np.testing.assert_allclose(out["w"], wa, rtol=1e-12, atol=1e-12)
        # stored basis: normalised residuals, mutually orthogonal
        V = out["V"]
        assert V.shape == (n, k)
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-8)


def make_recycle(rng, H, s):
    n = H.shape[0]
    Ut = rng.standard_normal((n, s))
    U, C = qr_normalise(Ut, H @ Ut)
    return U, C


def test_rcg_invariants(rng):
    n, s = 40, 6
    H = spd(rng, n, 1e3)
    g = rng.standard_normal(n)
    U, C = make_recycle(rng, H, s)
    np.testing.assert_allclose(C.T @ C, np.eye(s), atol=1e-12)
    np.testing.assert_allclose(H @ U, C, atol=1e-10)
    w0 = rng.standard_normal(n)
    for k in [0, 1, 5, 12]:
        out = rcg(lambda v: H @ v, g, w0, U, C, tol=0.0, maxit=k)
        r = out["r"]
        # Galerkin condition on C and the exact residual identity g - H w = r
        assert np.linalg.norm(C.T @ r) < 1e-10 * np.linalg.norm(g)
        np.testing.assert_allclose(g - H @ out["w"], r, atol=1e-9 * np.linalg.norm(g))
        if k:
            V = out["V"]
            # CG residuals lose orthogonality in proportion to kappa * eps per step
            np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-6)
            assert np.abs(C.T @ V).max() < 1e-10


def test_rcg_galerkin_bruteforce(rng):
    """After k steps: w = w0 + U C^T r0 + V y + U z with
    (V^T P H P V) y = V^T P r0,  z = -C^T H V y,  P = I - C C^T,
    and V spans the Krylov space K_k(P H P, P r0)."""
    n, s, k = 30, 4, 6
    H = spd(rng, n, 1e2)
    g = rng.standard_normal(n)
    w0 = rng.standard_normal(n)
    U, C = make_recycle(rng, H, s)
    P = np.eye(n) - C @ C.T
    r0 = g - H @ w0
    pr0 = P @ r0
    K = np.stack([np.linalg.matrix_power(P @ H @ P, j) @ pr0 for j in range(k)], axis=1)
    V, _ = np.linalg.qr(K)
    y = np.linalg.solve(V.T @ P @ H @ P @ V, V.T @ pr0)
    z = -C.T @ H @ V @ y
    w_expect = w0 + U @ (C.T @ r0) + V @ y + U @ z
    out = rcg(lambda v: H @ v, g, w0, U, C, tol=0.0, maxit=k)
    np.testing.assert_allclose(out["w"], w_expect, rtol=1e-8, atol=1e-8)


def test_rcg_converges_faster_with_exact_invariant_subspace(rng):
    """Deflating the eigenvectors of the s smallest eigenvalues removes them from CG."""
    n, s = 60, 8
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.logspace(-4, -3, s), np.linspace(1, 2, n - s)])
    H = (Q * lam) @ Q.T
    g = rng.standard_normal(n)
    U, C = qr_normalise(Q[:, :s], H @ Q[:, :s])
    plain = rcg(lambda v: H @ v, g, np.zeros(n), None, None, tol=1e-10, maxit=1000)
    rec = rcg(lambda v: H @ v, g, np.zeros(n), U, C, tol=1e-10, maxit=1000)
    assert rec["iters"] < plain["iters"]
    assert rec["iters"] <= 20            # kappa of the deflated operator is 2
    np.testing.assert_allclose(rec["w"], np.linalg.solve(H, g), rtol=1e-6)


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_minres_is_krylov_least_squares(k, rng):
    n = 20
    H = spd(rng, n, 50)
    H[0, 0] = -H[0, 0]               # symmetric indefinite is allowed for MINRES
    H = 0.5 * (H + H.T)
    g = rng.standard_normal(n)
    w0 = rng.standard_normal(n)
    r0 = g - H @ w0
    Kr = np.stack([np.linalg.matrix_power(H, j) @ r0 for j in range(k)], axis=1)
    V, _ = np.linalg.qr(Kr)
    y, *_ = np.linalg.lstsq(H @ V, r0, rcond=None)
    out = minres(lambda v: H @ v, g, w0, 0.0, k)
    np.testing.assert_allclose(out["w"], w0 + V @ y, rtol=1e-7, atol=1e-8)
    assert abs(out["resid"] - np.linalg.norm(g - H @ out["w"])) < 1e-8
    np.testing.assert_allclose(out["r"], g - H @ out["w"], atol=1e-8)


@pytest.mark.parametrize("indefinite", [False, True])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_rminres_solves_coupled_least_squares(k, indefinite, rng):
    """RMINRES minimises ||r0 - H [V_k U] [y; z]|| (eq. (2.11)) over the augmented
    Krylov space of (I - C C^T) H, after the initial projection onto C; also for a symmetric
    indefinite H (the non-convex phi of Section 5.2), where C = H U, C^T C = I still holds."""
    n, s = 24, 3
    H = spd(rng, n, 30)
    if indefinite:
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.concatenate([-np.logspace(0, 1, 5), np.logspace(0, 1.5, n - 5)])
        H = (Q * lam) @ Q.T
    g = rng.standard_normal(n)
    w0 = rng.standard_normal(n)
    U, C = make_recycle(rng, H, s)
    P = np.eye(n) - C @ C.T
    r0 = g - H @ w0
    w1 = w0 + U @ (C.T @ r0)
    r1 = P @ r0
    Kr = np.stack([np.linalg.matrix_power(P @ H, j) @ r1 for j in range(k)], axis=1)
    V, _ = np.linalg.qr(Kr)
    B = H @ np.hstack([V, U])
    yz, *_ = np.linalg.lstsq(B, r1, rcond=None)
    w_expect = w1 + np.hstack([V, U]) @ yz
    out = rminres(lambda v: H @ v, g, w0, U, C, tol=0.0, maxit=k)
    np.testing.assert_allclose(out["w"], w_expect, rtol=1e-7, atol=1e-8)
    # Appendix A: the recurrence residual is the true residual
    np.testing.assert_allclose(out["r"], g - H @ out["w"], atol=1e-8)
    assert abs(out["resid"] - np.linalg.norm(out["r"])) < 1e-8
