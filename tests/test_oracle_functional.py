"""Pins for Phi, grad Phi, the Hessian action and J w (eqs. (1.1), (2.4)-(2.7), (5.1)).

Finite differences fix the derivatives, dense assembly from the explicit
operator matrices fixes H and J, and the Tikhonov special case (one 1x1
filter, phi = s^2) fixes the whole hypergradient by a closed form.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import operators as ops
from oracle.functional import LowerLevel, phi_fns
from oracle.krylov import cg
from oracle.lbfgs import lbfgs


def make_ll(rng, h=8, w=9, reg="foe", N=2, f=3, phi="charbonnier", radius=2):
    G = ops.gaussian_kernel(1.5, radius)
    y = rng.uniform(0, 1, (h, w))
    ll = LowerLevel(y, G, reg, N, f, phi, 0.01 if phi == "charbonnier" else 1.0, 1e-6)
    if reg == "tv":
        theta = np.array([-1.0])
    else:
        theta = np.zeros(ll.p)
        for j in range(N):
            theta[j * (f * f + 1)] = -1.0 + 0.3 * j
            theta[j * (f * f + 1) + 1:(j + 1) * (f * f + 1)] = 0.5 * rng.standard_normal(f * f)
    x = rng.uniform(0, 1, (h, w))
    return ll, theta, x


CASES = [("foe", "charbonnier", 3), ("foe", "charbonnier", 5), ("foe", "sq", 3),
         ("foe", "log1p", 3), ("tv", "charbonnier", 0)]


@pytest.mark.parametrize("kind", ["charbonnier", "sq", "log1p"])
def test_phi_derivatives_fd(kind):
    f, df, d2f = phi_fns(kind, 0.05)
    s = np.linspace(-2, 2, 41)
    h = 1e-5
    np.testing.assert_allclose(df(s), (f(s + h) - f(s - h)) / (2 * h), rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(d2f(s), (df(s + h) - df(s - h)) / (2 * h), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("reg,phi,f", CASES)
def test_gradient_fd(reg, phi, f, rng):
    ll, th, x = make_ll(rng, reg=reg, phi=phi, f=max(f, 1))
    d = rng.standard_normal(x.shape)
    h = 1e-6
    fd = (ll.value(x + h * d, th) - ll.value(x - h * d, th)) / (2 * h)
    an = float(np.sum(ll.grad(x, th) * d))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


@pytest.mark.parametrize("reg,phi,f", CASES)
def test_hvp_fd_and_dense(reg, phi, f, rng):
    ll, th, x = make_ll(rng, reg=reg, phi=phi, f=max(f, 1))
    v = rng.standard_normal(x.shape)
    h = 1e-6
    fd = (ll.grad(x + h * v, th) - ll.grad(x - h * v, th)) / (2 * h)
    hv = ll.hvp(x, th, v)
    assert np.linalg.norm(fd - hv) < 1e-6 * np.linalg.norm(hv)
    Hd = ll.dense_hessian(x, th)
    np.testing.assert_allclose(Hd @ v.reshape(-1), hv.reshape(-1), rtol=0,
                               atol=1e-12 * np.abs(hv).max())
    np.testing.assert_allclose(Hd, Hd.T, atol=1e-12 * np.abs(Hd).max())


@pytest.mark.parametrize("reg,phi,f", CASES)
def test_hessian_symmetry_matrix_free(reg, phi, f, rng):
    ll, th, x = make_ll(rng, reg=reg, phi=phi, f=max(f, 1))
    v = rng.standard_normal(x.shape)
    w = rng.standard_normal(x.shape)
    a = float(np.sum(v * ll.hvp(x, th, w)))
    b = float(np.sum(w * ll.hvp(x, th, v)))
    assert abs(a - b) < 1e-12 * (abs(a) + 1)


def test_hessian_spd_for_convex_phi(rng):
    for reg, phi in [("foe", "charbonnier"), ("tv", "charbonnier"), ("foe", "sq")]:
        ll, th, x = make_ll(rng, reg=reg, phi=phi)
        Hd = ll.dense_hessian(x, th)
        sla.cho_factor(Hd)          # raises if not positive definite
        assert np.linalg.eigvalsh(Hd)[0] >= 1e-6 * 0.999


@pytest.mark.parametrize("reg,phi,f", CASES)
def test_Jw_fd_of_mixed_derivative(reg, phi, f, rng):
    """J w = -d/dtheta <grad_x Phi(x, theta), w>: central differences in theta."""
    ll, th, x = make_ll(rng, reg=reg, phi=phi, f=max(f, 1))
    w = rng.standard_normal(x.shape)
    jw = ll.Jw(x, th, w)
    h = 1e-6
    fd = np.zeros(ll.p)
    for m in range(ll.p):
        e = np.zeros(ll.p)
        e[m] = h
        fd[m] = -(np.sum(ll.grad(x, th + e) * w) - np.sum(ll.grad(x, th - e) * w)) / (2 * h)
    np.testing.assert_allclose(jw, fd, rtol=1e-6, atol=1e-7 * np.abs(jw).max())


@pytest.mark.parametrize("reg,phi,f", CASES)
def test_Jw_matches_dense_J(reg, phi, f, rng):
    ll, th, x = make_ll(rng, reg=reg, phi=phi, f=max(f, 1))
    w = rng.standard_normal(x.shape)
    J = ll.dense_J(x, th)
    assert J.shape == (ll.p, ll.n)
    np.testing.assert_allclose(ll.Jw(x, th, w), J @ w.reshape(-1), rtol=1e-11,
                               atol=1e-12 * np.abs(J).max())


def test_alpha_component_closed_form(rng):
    """The log-weight component is exactly -<exp(alpha) phi'(K x), K w> (eq. (5.1))."""
    ll, th, x = make_ll(rng, N=3, f=3)
    w = rng.standard_normal(x.shape)
    jw = ll.Jw(x, th, w)
    alphas, ks = ll.split(th)
    for j in range(3):
        u = ops.correlate(x, ks[j])
        expect = -np.exp(alphas[j]) * np.sum((u / np.sqrt(u * u + ll.eps ** 2)) * ops.correlate(w, ks[j]))
        assert abs(jw[j * 10] - expect) < 1e-12 * max(1, abs(expect))


def test_tikhonov_hypergradient_closed_form(rng):
    """One 1x1 filter with phi(s) = s^2 turns Phi into Tikhonov:
    x^ = M^{-1} 2 A^T y, M = 2 A^T A + lam I, lam = 2 e^alpha k^2 + eps, and
    dL/dtheta_m = -(d lam / d theta_m) x^T M^{-1} (x^ - x*)   (textbook implicit derivative).
    The checker's L-BFGS + CG + J w pipeline must reproduce it."""
    h, w = 7, 6
    G = ops.gaussian_kernel(1.2, 2)
    y = rng.uniform(0, 1, (h, w))
    xs = rng.uniform(0, 1, (h, w))
    ll = LowerLevel(y, G, "foe", 1, 1, "sq", 1.0, 1e-6)
    al, k = -1.3, 0.8
    theta = np.array([al, k])
    A = ops.dense_correlation(G, h, w)
    lam = 2 * np.exp(al) * k * k + 1e-6
    M = 2 * A.T @ A + lam * np.eye(h * w)
    xhat_cf = np.linalg.solve(M, 2 * A.T @ y.reshape(-1))
    dlam = np.array([2 * np.exp(al) * k * k, 4 * np.exp(al) * k])
    hg_cf = -dlam * float(xhat_cf @ np.linalg.solve(M, xhat_cf - xs.reshape(-1)))

    xh, info = lbfgs(lambda v: ll.value(v.reshape(h, w), theta),
                     lambda v: ll.grad(v.reshape(h, w), theta).reshape(-1),
                     np.zeros(h * w), 1e-12)
    np.testing.assert_allclose(xh, xhat_cf, rtol=0, atol=1e-10)
    g = xh - xs.reshape(-1)
    wv, _, _ = cg(lambda v: ll.hvp(xh.reshape(h, w), theta, v.reshape(h, w)).reshape(-1),
                  g, np.zeros_like(g), 1e-14, 1000)
    hg = ll.Jw(xh.reshape(h, w), theta, wv.reshape(h, w))
    np.testing.assert_allclose(hg, hg_cf, rtol=1e-8)
