"""Seeded synthetic inputs for the bilevel imaging workloads.

This module draws random numbers and nothing else: ground-truth images,
noise realisations, blur widths and initial filter taps.  It holds none of
the method's arithmetic (no blur, no regulariser, no solver), so that both
the CUDA path and the FP64 checker can take their inputs from it without
sharing any computation.  The measurement ``y = A x* + noise`` is formed by
each side with its own operator (blur, or for inpainting the measured-pixel mask,
which is drawn here as input data).

Image model (piecewise-constant, Section 5 uses natural images; these are
stand-ins of the same size): six axis-aligned rectangles with corners drawn
uniformly, side lengths uniform in [H/8, H/2] (clipped to the image),
painted in order over a zero background, each with a value U[0, 1].

Filter initialisation (Section 5, eq. (5.1) parametrisation): per filter
one log-weight alpha_j = -3 followed by f*f taps drawn N(0, 0.1^2) and made
zero-mean once (the deconvolution workload uses the non-constant DCT basis
filters instead, as Section 5.2 does).  theta = [alpha_1, taps_1, ..., alpha_N, taps_N].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

ROOT_SEED = 20241208


@dataclass
class PairSpec:
    height: int
    width: int
    blur_sigma: float
    blur_radius: int
    noise_sigma: float
    keep: float = 0.0           # inpainting: fraction of measured pixels (0: blur operator)


@dataclass
class Workload:
    """One synthetic workload: pairs, regulariser shape and solver settings."""
    name: str
    pairs: List[PairSpec]
    reg: str                    # "tv" or "foe"
    n_filters: int = 0
    filter_size: int = 0
    phi: str = "charbonnier"
    phi_eps: float = 0.01
    l2_eps: float = 1e-6
    recycle_dim: int = 0
    precision: str = "fp32"     # "fp32" (FP32 stencils, FP64 reductions) or "fp64"
    x_star: List[np.ndarray] = field(default_factory=list)
    noise: List[np.ndarray] = field(default_factory=list)
    masks: List[Optional[np.ndarray]] = field(default_factory=list)   # uint8 per pair, None: blur
    theta0: np.ndarray = None

    @property
    def n_params(self) -> int:
        if self.reg == "tv":
            return 1
        return self.n_filters * (self.filter_size ** 2 + 1)

    @property
    def n_pixels(self) -> int:
        return sum(p.height * p.width for p in self.pairs)


def rectangles_image(rng: np.random.Generator, h: int, w: int, n_rect: int = 6) -> np.ndarray:
    img = np.zeros((h, w), dtype=np.float64)
    for _ in range(n_rect):
        i0 = int(rng.integers(0, h))
        j0 = int(rng.integers(0, w))
        lh = int(rng.integers(max(1, h // 8), max(2, h // 2) + 1))
        lw = int(rng.integers(max(1, w // 8), max(2, w // 2) + 1))
        val = float(rng.uniform(0.0, 1.0))
        img[i0:min(h, i0 + lh), j0:min(w, j0 + lw)] = val
    return img


def gaussian_noise(rng: np.random.Generator, h: int, w: int, sigma: float) -> np.ndarray:
    return sigma * rng.standard_normal((h, w))


def keep_mask(rng: np.random.Generator, h: int, w: int, keep: float) -> np.ndarray:
    """Random subsampling pattern: each pixel measured independently with probability `keep`."""
    return (rng.random((h, w)) < keep).astype(np.uint8)


def foe_theta_init(rng: np.random.Generator, n_filters: int, f: int,
                   alpha0: float = -3.0, std: float = 0.1) -> np.ndarray:
    theta = np.empty(n_filters * (f * f + 1), dtype=np.float64)
    for j in range(n_filters):
        taps = std * rng.standard_normal(f * f)
        taps -= taps.mean()
        base = j * (f * f + 1)
        theta[base] = alpha0
        theta[base + 1: base + 1 + f * f] = taps
    return theta


def _fill(wl: Workload, ss: np.random.SeedSequence) -> Workload:
    kids = ss.spawn(len(wl.pairs) + 1)
    for p, kid in zip(wl.pairs, kids[:-1]):
        rng = np.random.default_rng(kid)
        wl.x_star.append(rectangles_image(rng, p.height, p.width))
        wl.noise.append(gaussian_noise(rng, p.height, p.width, p.noise_sigma))
        wl.masks.append(keep_mask(rng, p.height, p.width, p.keep) if p.keep > 0 else None)
    rng = np.random.default_rng(kids[-1])
    if wl.reg == "tv":
        wl.theta0 = np.array([-3.0])
    else:
        wl.theta0 = foe_theta_init(rng, wl.n_filters, wl.filter_size)
    return wl


def _cfg_seed(index: int) -> np.random.SeedSequence:
    return np.random.SeedSequence(ROOT_SEED).spawn(8)[index]


def tv_32() -> Workload:
    """Single 32x32 image, TV regulariser, all FP64."""
    wl = Workload("tv32_fp64", [PairSpec(32, 32, 1.5, 2, 0.01)], reg="tv",
                  precision="fp64")
    return _fill(wl, _cfg_seed(0))


def foe_256() -> Workload:
    """Single 256x256 image, FoE with 8 5x5 filters (p = 208), recycle dim 20."""
    wl = Workload("foe256_n8f5", [PairSpec(256, 256, 1.5, 2, 0.02)], reg="foe",
                  n_filters=8, filter_size=5, recycle_dim=20)
    return _fill(wl, _cfg_seed(1))


def batch_64(replica: int = 0) -> Workload:
    """64 pairs of uneven square sizes, FoE with 16 5x5 filters (p = 416), recycle dim 16.

    replica > 0 draws an independent batch of the same recipe (one per data-parallel rank)."""
    ss = _cfg_seed(2) if replica == 0 else np.random.SeedSequence([ROOT_SEED, 2, replica])
    meta_ss, data_ss = ss.spawn(2)
    rng = np.random.default_rng(meta_ss)
    sides = [128, 192, 256, 384, 512]
    pairs = []
    for _ in range(64):
        side = int(sides[int(rng.integers(0, len(sides)))])
        pairs.append(PairSpec(side, side, float(rng.uniform(1.0, 2.5)), 4,
                              float(rng.uniform(0.005, 0.03))))
    wl = Workload("batch64_foe_n16f5", pairs, reg="foe", n_filters=16, filter_size=5,
                  recycle_dim=16)
    return _fill(wl, data_ss)


def batch_1024() -> Workload:
    """8 images of 1024x1024, FoE with 24 7x7 filters (p = 1200)."""
    wl = Workload("batch8_1024_foe_n24f7", [PairSpec(1024, 1024, 1.5, 2, 0.02)] * 8,
                  reg="foe", n_filters=24, filter_size=7, recycle_dim=16)
    return _fill(wl, _cfg_seed(3))


def large_2048() -> Workload:
    """Single 2048x2048 image, 9x9 blur sigma 3, FoE with 48 7x7 filters, recycle dim 50."""
    wl = Workload("large2048_foe_n48f7", [PairSpec(2048, 2048, 3.0, 4, 0.01)], reg="foe",
                  n_filters=48, filter_size=7, recycle_dim=50)
    return _fill(wl, _cfg_seed(4))


def small_foe(h: int, w: int, n_filters: int = 3, f: int = 5, blur_radius: int = 2,
              blur_sigma: float = 1.5, noise_sigma: float = 0.02, seed: int = 0,
              n_pairs: int = 1) -> Workload:
    """Small FoE workload for tests (several tiles, ragged tails)."""
    pairs = [PairSpec(h, w, blur_sigma, blur_radius, noise_sigma)] * n_pairs
    wl = Workload(f"foe{h}x{w}_n{n_filters}f{f}", pairs, reg="foe", n_filters=n_filters,
                  filter_size=f, recycle_dim=8)
    return _fill(wl, np.random.SeedSequence([ROOT_SEED, 7, seed]))


def uneven_foe(sizes, n_filters: int = 4, f: int = 5, blur_radius: int = 4, seed: int = 0) -> Workload:
    """Several pairs of the given (h, w) sizes, per-pair blur and noise drawn like the batch workload."""
    ss = np.random.SeedSequence([ROOT_SEED, 11, seed])
    meta_ss, data_ss = ss.spawn(2)
    rng = np.random.default_rng(meta_ss)
    pairs = [PairSpec(h, w, float(rng.uniform(1.0, 2.5)), blur_radius,
                      float(rng.uniform(0.005, 0.03))) for (h, w) in sizes]
    wl = Workload("uneven_foe", pairs, reg="foe", n_filters=n_filters, filter_size=f,
                  recycle_dim=8)
    return _fill(wl, data_ss)


def dct_filters(n_filters: int, f: int) -> np.ndarray:
    """The non-constant 2-D DCT-II basis filters of size f x f (unit l2 norm), ordered by frequency
    pair (u, v) row-major, (0, 0) left out: Section 5.2 initialises the FoE filters with them."""
    out = []
    a = np.arange(f)
    for u in range(f):
        for v in range(f):
            if u == 0 and v == 0:
                continue
            k = np.outer(np.cos(np.pi * (2 * a + 1) * u / (2 * f)), np.cos(np.pi * (2 * a + 1) * v / (2 * f)))
            out.append(k / np.linalg.norm(k))
    if n_filters > len(out):
        raise ValueError("more filters than non-constant DCT basis functions")
    return np.stack(out[:n_filters])


def deconv_batch(n_pairs: int = 512, side: int = 64, blur_sigma: float = 3.0, blur_radius: int = 4,
                 noise_sigma: float = 0.08, n_filters: int = 24, f: int = 5, seed: int = 0) -> Workload:
    """Deconvolution pairs shaped like Section 5.2's experiment (512 crops of 64 x 64, Gaussian blur
    sigma 3 truncated to 9 x 9, noise, 24 learned 5 x 5 filters with phi = log(1 + s^2), the filters
    initialised with the non-constant DCT basis and alpha_j = -3)."""
    pairs = [PairSpec(side, side, blur_sigma, blur_radius, noise_sigma)] * n_pairs
    wl = Workload(f"deconv{n_pairs}x{side}_n{n_filters}f{f}", pairs, reg="foe", n_filters=n_filters,
                  filter_size=f, phi="log1p", recycle_dim=16)
    wl = _fill(wl, np.random.SeedSequence([ROOT_SEED, 19, seed]))
    taps = dct_filters(n_filters, f)
    theta = np.empty(n_filters * (f * f + 1))
    for j in range(n_filters):
        theta[j * (f * f + 1)] = -3.0
        theta[j * (f * f + 1) + 1:(j + 1) * (f * f + 1)] = taps[j].ravel()
    wl.theta0 = theta
    return wl


def inpaint_batch(n_pairs: int = 1024, side: int = 28, keep: float = 0.3, noise_sigma: float = 0.1,
                  n_filters: int = 3, f: int = 5, seed: int = 0) -> Workload:
    """Inpainting pairs shaped like Section 5.1's experiment (28 x 28 images, 30 % of the pixels
    measured, heavy noise, 3 learned 5 x 5 filters with phi = s^2), batched over many pairs."""
    pairs = [PairSpec(side, side, 1.0, 0, noise_sigma, keep)] * n_pairs
    wl = Workload(f"inpaint{n_pairs}x{side}_n{n_filters}f{f}", pairs, reg="foe", n_filters=n_filters,
                  filter_size=f, phi="sq", recycle_dim=30)
    return _fill(wl, np.random.SeedSequence([ROOT_SEED, 13, seed]))


WORKLOADS = {
    "tv32_fp64": tv_32,
    "foe256_n8f5": foe_256,
    "batch64_foe_n16f5": batch_64,
    "batch8_1024_foe_n24f7": batch_1024,
    "large2048_foe_n48f7": large_2048,
    "inpaint1024x28_n3f5": inpaint_batch,
    "deconv512x64_n24f5": deconv_batch,
}


def random_vectors(n: int, k: int, seed: int) -> np.ndarray:
    """k seeded standard-normal vectors of length n (test probes), shape (k, n)."""
    return np.random.default_rng(np.random.SeedSequence([ROOT_SEED, 99, seed])).standard_normal((k, n))
