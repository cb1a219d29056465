"""The crop evaluations used by the full-size parity tests equal the checker's full-image
results (so the sampled comparisons at full size are exact), and a margin one short of the
stated dependency radius is detected (the check is sharp)."""
import numpy as np
import pytest

from oracle import operators as ops
from oracle.functional import LowerLevel
from tests import crops


def level(rng, reg, f, N, rb, mask=False, h=61, w=74, phi="charbonnier"):
    y = rng.uniform(0, 1, (h, w))
    m = (rng.random((h, w)) < 0.3).astype(np.uint8) if mask else None
    G = None if mask else ops.gaussian_kernel(1.7, rb)
    ll = LowerLevel(y, G, reg, N, f, phi, 0.01 if phi == "charbonnier" else 1.0, 1e-6, mask=m)
    if reg == "tv":
        th = np.array([-1.0])
    else:
        th = np.zeros(ll.p)
        for j in range(N):
            th[j * (f * f + 1)] = -0.5 + 0.2 * j
            th[j * (f * f + 1) + 1:(j + 1) * (f * f + 1)] = 0.7 * rng.standard_normal(f * f)
    return ll, th


CASES = [("foe", 7, 3, 4, False, "charbonnier"), ("foe", 5, 4, 2, False, "log1p"), ("foe", 5, 2, 0, True, "sq"),
         ("foe", 3, 2, 1, False, "charbonnier"), ("tv", 0, 0, 3, False, "charbonnier")]


@pytest.mark.parametrize("reg,f,N,rb,mask,phi", CASES)
def test_hvp_crops_equal_full_image(reg, f, N, rb, mask, phi, rng):
    ll, th = level(rng, reg, f, N, rb, mask, phi=phi)
    x = rng.uniform(-0.2, 1.2, (ll.h, ll.w))
    v = rng.standard_normal((ll.h, ll.w))
    full = ll.hvp(x, th, v)
    pix = crops.sample_pixels(rng, ll.h, ll.w, 40)
    got = crops.hvp_at(ll, x, th, v, pix)
    ref = np.array([full[i, j] for i, j in pix])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(full))
    # one pixel short of the dependency radius: some interior pixel changes
    M = crops.hvp_margin(ll)
    interior = [(i, j) for i, j in pix if M <= i < ll.h - M and M <= j < ll.w - M]
    short = crops.hvp_at(ll, x, th, v, interior, margin=M - 1)
    ref_i = np.array([full[i, j] for i, j in interior])
    assert np.max(np.abs(short - ref_i)) > 1e-9 * np.max(np.abs(full))


@pytest.mark.parametrize("reg,f,N,rb,mask,phi", CASES)
def test_jw_patches_equal_full_image(reg, f, N, rb, mask, phi, rng):
    ll, th = level(rng, reg, f, N, rb, mask, phi=phi)
    x = rng.uniform(-0.2, 1.2, (ll.h, ll.w))
    for patch in crops.patches(ll.h, ll.w):
        w = crops.patch_vector(rng, ll.h, ll.w, patch)
        full = ll.Jw(x, th, w)
        got = crops.jw_patch(ll, x, th, w, patch)
        assert np.linalg.norm(got - full) <= 1e-12 * np.linalg.norm(full)
    # the interior patch with one pixel too little margin gives a different J w
    patch = crops.patches(ll.h, ll.w)[2]
    w = crops.patch_vector(rng, ll.h, ll.w, patch)
    short = crops.jw_patch(ll, x, th, w, patch, margin=crops.jw_margin(ll) - 1)
    full = ll.Jw(x, th, w)
    assert np.linalg.norm(short - full) > 1e-9 * np.linalg.norm(full)
