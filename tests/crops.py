"""Exact checker values at sampled points of full-size images, computed on small crops.

The checker's full-image operators take minutes at 1024^2 and 2048^2, so the full-size parity
tests compare sampled outputs, each evaluated exactly on a crop:

  Hessian action.  (H v)[p] is a sum of separate terms: the data term A (A v) reads v within
  2 r_b of p (the intermediate A v kept on the image; 0 for an inpainting mask), and each filter
  term K_j^T (d_j (K_j v)) reads (K_j v) and d_j = e^{alpha_j} phi''(K_j x^) at q within r_f of
  p, so v and x^ within 2 r_f of p (eq. (5.1)); TV reads v and x^ within 1 (a forward difference
  and its adjoint).  A crop reaching max(data radius, regulariser radius) from p on every side
  the image continues past evaluates (H v)[p] exactly: where the crop meets the real border, its
  zero boundary is the image's.

  J w for a w supported on a patch.  Every term of J w (eq. (2.7) with eq. (5.1)) carries
  (K_j w)_p or w_{p+o}, non-zero only within r_f of the patch, times phi'(u_p) or phi''(u_p)
  x^_{p+o}, which read x^ within 2 r_f of the patch; the patch grown by 2 r_f (1 for TV) gives
  J w exactly.
"""
from __future__ import annotations

import numpy as np

from oracle.functional import LowerLevel


def crop_level(ll: LowerLevel, i0: int, i1: int, j0: int, j1: int) -> LowerLevel:
    return LowerLevel(ll.y[i0:i1, j0:j1], ll.G, ll.reg, ll.N, ll.f, ll.phi_kind, ll.eps, ll.l2,
                      mask=None if ll.mask is None else ll.mask[i0:i1, j0:j1])


def _reg_radius(ll: LowerLevel) -> int:
    return 1 if ll.reg == "tv" else 2 * (ll.f // 2)


def hvp_margin(ll: LowerLevel) -> int:
    rb = 0 if ll.mask is not None else ll.G.shape[0] // 2
    return max(2 * rb, _reg_radius(ll))


def jw_margin(ll: LowerLevel) -> int:
    return _reg_radius(ll)


def _window(c, lo_margin, hi_margin, n):
    return max(0, c - lo_margin), min(n, c + hi_margin)


def hvp_at(ll: LowerLevel, x, theta, v, pixels, margin=None):
    """(H v)[p] for each (i, j) in pixels, each from the crop p +- margin (default: exact)."""
    M = hvp_margin(ll) if margin is None else margin
    out = []
    for i, j in pixels:
        i0, i1 = _window(i, M, M + 1, ll.h)
        j0, j1 = _window(j, M, M + 1, ll.w)
        hv = crop_level(ll, i0, i1, j0, j1).hvp(x[i0:i1, j0:j1], theta, v[i0:i1, j0:j1])
        out.append(hv[i - i0, j - j0])
    return np.array(out)


def jw_patch(ll: LowerLevel, x, theta, w, patch, margin=None):
    """J w for w zero outside patch = (i0, i1, j0, j1), from the patch grown by the margin."""
    M = jw_margin(ll) if margin is None else margin
    pi0, pi1, pj0, pj1 = patch
    i0, i1 = max(0, pi0 - M), min(ll.h, pi1 + M)
    j0, j1 = max(0, pj0 - M), min(ll.w, pj1 + M)
    return crop_level(ll, i0, i1, j0, j1).Jw(x[i0:i1, j0:j1], theta, w[i0:i1, j0:j1])


def sample_pixels(rng, h, w, n_random):
    """The four corners, points on each edge, points just inside the blur and filter halos, and
    n_random uniform interior points (duplicates removed, order kept)."""
    pts = [(0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1), (0, w // 2), (h - 1, w // 3), (h // 2, 0),
           (h // 3, w - 1), (min(h - 1, 5), min(w - 1, 6)), (max(0, h - 7), max(0, w - 4))]
    pts += [(int(rng.integers(0, h)), int(rng.integers(0, w))) for _ in range(n_random)]
    seen, out = set(), []
    for p in pts:
        if p not in seen:
            seen.add(p)
            out.append(p)
    return out


def patches(h, w, size=12):
    """Three patches of w's support: at the top-left corner, on the right edge, in the interior."""
    s_h, s_w = min(size, h), min(size, w)
    return [(0, s_h, 0, s_w), (h // 2, min(h, h // 2 + s_h), w - s_w, w),
            (h // 3, min(h, h // 3 + s_h), w // 3, min(w, w // 3 + s_w))]


def patch_vector(rng, h, w, patch):
    v = np.zeros((h, w))
    i0, i1, j0, j1 = patch
    v[i0:i1, j0:j1] = rng.standard_normal((i1 - i0, j1 - j0))
    return v
