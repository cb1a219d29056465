"""Pins for the checker's linear operators (Section 5, eq. (5.1) and the blur of Section 5.2).

Each shift-based operator is compared with a dense matrix assembled by explicit
index loops (independent code) and with its adjoint identity.
"""
import numpy as np
import pytest

from oracle import operators as ops


@pytest.mark.parametrize("f", [3, 5, 7])
@pytest.mark.parametrize("shape", [(7, 9), (6, 6), (1, 8), (9, 1)])
def test_correlation_matches_dense(f, shape, rng):
    h, w = shape
    k = rng.standard_normal((f, f))
    x = rng.standard_normal(shape)
    u = rng.standard_normal(shape)
    M = ops.dense_correlation(k, h, w)
    np.testing.assert_allclose(ops.correlate(x, k).reshape(-1), M @ x.reshape(-1), rtol=0, atol=1e-13)
    np.testing.assert_allclose(ops.correlate_adjoint(u, k).reshape(-1), M.T @ u.reshape(-1),
                               rtol=0, atol=1e-13)


def test_correlation_adjoint_identity(rng):
    k = rng.standard_normal((5, 5))
    x = rng.standard_normal((13, 11))
    u = rng.standard_normal((13, 11))
    lhs = np.sum(ops.correlate(x, k) * u)
    rhs = np.sum(x * ops.correlate_adjoint(u, k))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_correlation_centre_tap_is_identity(rng):
    k = np.zeros((5, 5))
    k[2, 2] = 1.0
    x = rng.standard_normal((6, 7))
    np.testing.assert_array_equal(ops.correlate(x, k), x)
    k = np.zeros((3, 3))
    k[2, 1] = 1.0                   # o = (+1, 0): (Kx)[i, j] = x[i + 1, j]
    y = ops.correlate(x, k)
    np.testing.assert_array_equal(y[:-1], x[1:])
    np.testing.assert_array_equal(y[-1], 0.0)


@pytest.mark.parametrize("sigma,radius", [(1.5, 2), (3.0, 4), (1.0, 4), (2.5, 4)])
def test_gaussian_kernel(sigma, radius):
    G = ops.gaussian_kernel(sigma, radius)
    assert G.shape == (2 * radius + 1,) * 2
    assert abs(G.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(G, G.T, atol=0)
    np.testing.assert_allclose(G, G[::-1, ::-1], atol=0)
    # separable: G = g g^T with the normalised 1-D Gaussian (closed form)
    a = np.arange(-radius, radius + 1)
    g = np.exp(-a ** 2 / (2 * sigma ** 2))
    g /= g.sum()
    np.testing.assert_allclose(G, np.outer(g, g), rtol=1e-14, atol=1e-17)
    # the ratio of the centre to a neighbour is exp(1 / (2 sigma^2))
    assert abs(G[radius, radius] / G[radius, radius + 1] - np.exp(1 / (2 * sigma ** 2))) < 1e-12


def test_blur_preserves_constants_in_interior():
    G = ops.gaussian_kernel(1.5, 2)
    x = np.full((12, 12), 0.7)
    y = ops.blur(x, G)
    np.testing.assert_allclose(y[2:-2, 2:-2], 0.7, rtol=1e-14)
    assert y[0, 0] < 0.7            # zero boundary truncates the support


def test_blur_self_adjoint(rng):
    G = ops.gaussian_kernel(2.0, 3)
    A = ops.dense_correlation(G, 8, 10)
    np.testing.assert_allclose(A, A.T, atol=1e-16)


@pytest.mark.parametrize("shape", [(5, 7), (1, 6), (6, 1)])
def test_forward_differences(shape, rng):
    h, w = shape
    x = rng.standard_normal(shape)
    D = ops.dense_grad(h, w)
    d = ops.grad_fwd(x)
    np.testing.assert_allclose(d.reshape(-1), D @ x.reshape(-1), atol=1e-14)
    u = rng.standard_normal((2, h, w))
    np.testing.assert_allclose(ops.grad_adj(u).reshape(-1), D.T @ u.reshape(-1), atol=1e-14)
    # Neumann convention: the last row's vertical and last column's horizontal differences vanish
    assert np.all(d[0, -1, :] == 0) and np.all(d[1, :, -1] == 0)
    # constants have zero gradient
    assert np.all(ops.grad_fwd(np.ones(shape)) == 0)


def test_dense_shift(rng):
    x = rng.standard_normal((5, 6))
    for a, b in [(1, 0), (0, -2), (-1, 3), (2, 2)]:
        S = ops.dense_shift(a, b, 5, 6)
        np.testing.assert_array_equal(ops.shift(x, a, b).reshape(-1), S @ x.reshape(-1))
