"""Pins for the inpainting forward operator of Section 5.1 (A keeps a random subset of pixels):
the definition by brute force, finite differences of Phi and grad Phi, the dense Hessian, the
quadratic (phi = s^2) lower level against normal equations assembled by explicit loops, and the
hypergradient against central differences of the upper loss."""
import numpy as np
import pytest

from oracle.functional import LowerLevel


def masked_ll(rng, h=9, w=11, reg="foe", N=2, f=3, phi="sq", keep=0.3):
    m = (rng.random((h, w)) < keep).astype(np.uint8)
    xs = rng.uniform(0, 1, (h, w))
    y = m * (xs + 0.1 * rng.standard_normal((h, w)))
    eps = 0.01 if phi == "charbonnier" else 1.0
    ll = LowerLevel(y, None, reg, N, f, phi, eps, 1e-6, mask=m)
    if reg == "tv":
        th = np.array([-1.0])
    else:
        th = np.zeros(ll.p)
        for j in range(N):
            th[j * (f * f + 1)] = -1.0 + 0.3 * j
            th[j * (f * f + 1) + 1:(j + 1) * (f * f + 1)] = 0.5 * rng.standard_normal(f * f)
    return ll, th, m, xs


def test_mask_operator_definition(rng):
    ll, th, m, _ = masked_ll(rng)
    x = rng.standard_normal(m.shape)
    Ax = ll.A(x)
    for i in range(m.shape[0]):
        for j in range(m.shape[1]):
            assert Ax[i, j] == (x[i, j] if m[i, j] else 0.0)
    u = rng.standard_normal(m.shape)
    assert abs(np.sum(ll.A(x) * u) - np.sum(x * ll.At(u))) < 1e-12
    np.testing.assert_array_equal(np.diag(ll.dense_A()), m.reshape(-1).astype(float))
    assert np.count_nonzero(ll.dense_A() - np.diag(np.diag(ll.dense_A()))) == 0


@pytest.mark.parametrize("reg,phi", [("foe", "sq"), ("foe", "charbonnier"), ("foe", "log1p"), ("tv", "charbonnier")])
def test_masked_gradient_and_hvp_fd(reg, phi, rng):
    ll, th, m, _ = masked_ll(rng, reg=reg, phi=phi)
    x = rng.uniform(0, 1, m.shape)
    d = rng.standard_normal(m.shape)
    h = 1e-6
    fd = (ll.value(x + h * d, th) - ll.value(x - h * d, th)) / (2 * h)
    an = float(np.sum(ll.grad(x, th) * d))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
    fdh = (ll.grad(x + h * d, th) - ll.grad(x - h * d, th)) / (2 * h)
    hv = ll.hvp(x, th, d)
    assert np.linalg.norm(fdh - hv) < 1e-5 * max(1.0, np.linalg.norm(hv))
    H = ll.dense_hessian(x, th)
    assert np.linalg.norm(H @ d.reshape(-1) - hv.reshape(-1)) < 1e-10 * np.linalg.norm(hv)


def brute_correlation_matrix(k, h, w):
    """(K x)[p] = sum_o k[o] x[p + o], zero outside, by explicit loops (independent of the
    checker's shift helpers)."""
    r = k.shape[0] // 2
    K = np.zeros((h * w, h * w))
    for i in range(h):
        for j in range(w):
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < h and 0 <= jj < w:
                        K[i * w + j, ii * w + jj] += k[a + r, b + r]
    return K


def test_quadratic_inpainting_normal_equations(rng):
    """phi = s^2: grad Phi = 2 M (x - y) + l2 x + 2 sum_j e^{alpha_j} K_j^T K_j x = 0 is linear; the
    checker's gradient vanishes at the normal-equation solution built by explicit loops."""
    ll, th, m, _ = masked_ll(rng, h=7, w=8, phi="sq")
    n = ll.n
    alphas, ks = ll.split(th)
    M = np.diag(m.reshape(-1).astype(float))
    Hn = 2 * M + ll.l2 * np.eye(n)
    for al, k in zip(alphas, ks):
        K = brute_correlation_matrix(k, ll.h, ll.w)
        Hn += 2 * np.exp(al) * K.T @ K
    x = np.linalg.solve(Hn, 2 * M @ ll.y.reshape(-1)).reshape(ll.h, ll.w)
    g = ll.grad(x, th)
    assert np.linalg.norm(g) < 1e-10 * np.linalg.norm(2 * M @ ll.y.reshape(-1))
    np.testing.assert_allclose(ll.dense_hessian(x, th), Hn, atol=1e-12)


def test_masked_hypergradient_fd(rng):
    """Quadratic lower level (exact solves by the dense normal equations): J w with H w = x^ - x*
    matches central differences of 1/2 ||x^(theta) - x*||^2."""
    ll, th, m, xs = masked_ll(rng, h=7, w=8, phi="sq")

    def lower(theta):
        H = ll.dense_hessian(np.zeros((ll.h, ll.w)), theta)   # phi = s^2: H independent of x
        return np.linalg.solve(H, 2 * ll.A(ll.y).reshape(-1)).reshape(ll.h, ll.w)

    def loss(theta):
        return 0.5 * float(np.sum((lower(theta) - xs) ** 2))

    xh = lower(th)
    w = np.linalg.solve(ll.dense_hessian(xh, th), (xh - xs).reshape(-1)).reshape(ll.h, ll.w)
    hg = ll.Jw(xh, th, w)
    for _ in range(3):
        d = rng.standard_normal(ll.p)
        d /= np.linalg.norm(d)
        hh = 1e-5
        fd = (loss(th + hh * d) - loss(th - hh * d)) / (2 * hh)
        assert abs(fd - hg @ d) < 1e-6 * max(1.0, abs(hg @ d))


def test_dct_filters_are_an_orthonormal_zero_mean_basis():
    """The 24 non-constant 5 x 5 DCT-II filters of the deconvolution workload: orthonormal, zero
    mean, and with the constant filter they span all 5 x 5 filters."""
    from paper_2412_08264_gb300 import synth
    B = synth.dct_filters(24, 5).reshape(24, 25)
    np.testing.assert_allclose(B @ B.T, np.eye(24), atol=1e-12)
    np.testing.assert_allclose(B.sum(axis=1), 0.0, atol=1e-12)
    full = np.vstack([np.full(25, 0.2), B])
    assert np.linalg.matrix_rank(full) == 25
