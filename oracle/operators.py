"""Linear image operators in FP64 (Section 5, eq. (5.1); blur of Section 5.2).

Images are (H, W) arrays, pixel p = (i, j).  Every operator uses a zero
boundary and "same" output size.  Convolution in eq. (5.1) is read as
correlation with centred taps: (K x)[p] = sum_o k[o] x[p + o], o in
[-r, r]^2 (a filter flip only relabels theta).
"""
from __future__ import annotations

import numpy as np


def shift(x: np.ndarray, a: int, b: int) -> np.ndarray:
    """y[i, j] = x[i + a, j + b], zero where (i + a, j + b) is outside the image."""
    h, w = x.shape
    y = np.zeros_like(x)
    i0, i1 = max(0, -a), min(h, h - a)
    j0, j1 = max(0, -b), min(w, w - b)
    if i0 < i1 and j0 < j1:
        y[i0:i1, j0:j1] = x[i0 + a:i1 + a, j0 + b:j1 + b]
    return y


def correlate(x: np.ndarray, k: np.ndarray) -> np.ndarray:
    """(K x)[p] = sum_o k[o] x[p + o]; k is (f, f) with f = 2r + 1, k[r + a, r + b] = k[o=(a, b)]."""
    f = k.shape[0]
    r = f // 2
    out = np.zeros_like(x)
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            out += k[r + a, r + b] * shift(x, a, b)
    return out


def correlate_adjoint(u: np.ndarray, k: np.ndarray) -> np.ndarray:
    """(K^T u)[q] = sum_o k[o] u[q - o]."""
    f = k.shape[0]
    r = f // 2
    out = np.zeros_like(u)
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            out += k[r + a, r + b] * shift(u, -a, -b)
    return out


def gaussian_kernel(sigma: float, radius: int) -> np.ndarray:
    """G[a, b] proportional to exp(-(a^2 + b^2) / (2 sigma^2)) on [-radius, radius]^2, summing to 1."""
    a = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def blur(x: np.ndarray, G: np.ndarray) -> np.ndarray:
    """A x with A the Gaussian blur; G is symmetric so A^T = A."""
    return correlate(x, G)


def blur_adjoint(u: np.ndarray, G: np.ndarray) -> np.ndarray:
    return correlate_adjoint(u, G)


def grad_fwd(x: np.ndarray) -> np.ndarray:
    """D x: forward differences, zero in the last row (vertical) / last column (horizontal).

    Returns an array (2, H, W): [0] = x[i+1, j] - x[i, j], [1] = x[i, j+1] - x[i, j].
    """
    d = np.zeros((2,) + x.shape, dtype=x.dtype)
    d[0, :-1, :] = x[1:, :] - x[:-1, :]
    d[1, :, :-1] = x[:, 1:] - x[:, :-1]
    return d


def grad_adj(d: np.ndarray) -> np.ndarray:
    """D^T applied to a field (2, H, W)."""
    out = np.zeros(d.shape[1:], dtype=d.dtype)
    out[1:, :] += d[0, :-1, :]
    out[:-1, :] -= d[0, :-1, :]
    out[:, 1:] += d[1, :, :-1]
    out[:, :-1] -= d[1, :, :-1]
    return out


# Dense matrices, assembled entry by entry with explicit index loops.  They
# share no code with the shift-based operators above and pin them in tests.

def dense_correlation(k: np.ndarray, h: int, w: int) -> np.ndarray:
    f = k.shape[0]
    r = f // 2
    n = h * w
    M = np.zeros((n, n))
    for i in range(h):
        for j in range(w):
            p = i * w + j
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < h and 0 <= jj < w:
                        M[p, ii * w + jj] += k[r + a, r + b]
    return M


def dense_grad(h: int, w: int) -> np.ndarray:
    """Rows 0..n-1: vertical differences, rows n..2n-1: horizontal differences."""
    n = h * w
    D = np.zeros((2 * n, n))
    for i in range(h):
        for j in range(w):
            p = i * w + j
            if i + 1 < h:
                D[p, p + w] = 1.0
                D[p, p] = -1.0
            if j + 1 < w:
                D[n + p, p + 1] = 1.0
                D[n + p, p] = -1.0
    return D


def dense_shift(a: int, b: int, h: int, w: int) -> np.ndarray:
    """S with (S x)[p] = x[p + (a, b)], zero outside."""
    n = h * w
    S = np.zeros((n, n))
    for i in range(h):
        for j in range(w):
            ii, jj = i + a, j + b
            if 0 <= ii < h and 0 <= jj < w:
                S[i * w + j, ii * w + jj] = 1.0
    return S
