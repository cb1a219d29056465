"""GPU parity of the inpainting forward operator (Section 5.1: A keeps a random subset of the
pixels) against the FP64 checker: bl_forward, the Hessian action, the gradient and value, a TV
problem (direct kernels), and the whole FP32 hypergradient.  Batches mix inpainting and blur pairs
so the per-pair operator choice is exercised inside one launch; sizes span several tiles with
ragged tails.  Tolerances as for the blur operator: 1e-5 (FP32), 1e-12 (FP64), 1e-4 on
hypergradients."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from oracle.krylov import cg
from tests.gpu_util import DEV, make, packed, r32, rel, split

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def mixed_workload(seed=0, phi="sq", reg="foe", widths4=False):
    """Three inpainting pairs (30 % kept) and one blur pair (widths4: every width a multiple of 4, so
    the FP32 Hessian action runs the TMA-staged kernel)."""
    if widths4:
        wl = synth.Workload("mixed_inpaint4", [synth.PairSpec(28, 28, 1.0, 0, 0.1, 0.3),
                                               synth.PairSpec(70, 132, 1.0, 0, 0.1, 0.3),
                                               synth.PairSpec(37, 44, 1.0, 0, 0.1, 0.5),
                                               synth.PairSpec(40, 52, 1.7, 3, 0.02)],
                            reg="foe", n_filters=3, filter_size=5, phi=phi, recycle_dim=8)
    elif reg == "tv":
        wl = synth.tv_32()
        wl.pairs = [synth.PairSpec(28, 28, 1.0, 0, 0.1, 0.3), synth.PairSpec(70, 131, 1.0, 0, 0.1, 0.3),
                    synth.PairSpec(13, 21, 1.2, 1, 0.01)]
    else:
        wl = synth.Workload("mixed_inpaint", [synth.PairSpec(28, 28, 1.0, 0, 0.1, 0.3),
                                              synth.PairSpec(70, 131, 1.0, 0, 0.1, 0.3),
                                              synth.PairSpec(37, 45, 1.0, 0, 0.1, 0.5),
                                              synth.PairSpec(40, 52, 1.7, 3, 0.02)],
                            reg="foe", n_filters=3, filter_size=5, phi=phi, recycle_dim=8)
    wl.x_star, wl.noise, wl.masks = [], [], []
    return synth._fill(wl, np.random.SeedSequence([synth.ROOT_SEED, 17, seed]))


def point(wl, rng):
    return [r32(np.clip(x + 0.05 * rng.standard_normal(x.shape), -0.2, 1.2)) for x in wl.x_star]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_forward_mask(precision):
    wl = mixed_workload()
    assert sum(m is not None for m in wl.masks) == 3
    P, prob, dt = make(wl, precision)
    out = split(P.forward(packed(prob.x_star, dt)), P.sizes)
    for got, xs, ll in zip(out, prob.x_star, prob.lowers):
        assert rel(got, ll.A(xs)) < TOL[precision]
        if ll.mask is not None:
            assert np.all(got[ll.mask == 0] == 0)


@pytest.mark.parametrize("precision, widths4", [("fp32", False), ("fp64", False), ("fp32", True)],
                         ids=["fp32", "fp64", "fp32-tma"])
@pytest.mark.parametrize("phi", ["sq", "charbonnier"])
def test_hvp_gradient_value_parity_mask(precision, phi, widths4):
    wl = mixed_workload(seed=1, phi=phi, widths4=widths4)
    P, prob, dt = make(wl, precision)
    assert P.hvp_tma() == widths4
    rng = np.random.default_rng(1)
    xs = point(wl, rng)
    th0 = r32(wl.theta0) if precision == "fp32" else wl.theta0
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    g, vals = P.gradient(theta, packed(xs, dt))
    g = split(g, P.sizes)
    vals = vals.cpu().numpy()
    for k, ll in enumerate(prob.lowers):
        assert rel(g[k], ll.grad(xs[k], th0)) < TOL[precision], (k, rel(g[k], ll.grad(xs[k], th0)))
        assert abs(vals[k] - ll.value(xs[k], th0)) < TOL[precision] * abs(ll.value(xs[k], th0))
    P.set_point(theta, packed(xs, dt))
    vs = [r32(rng.standard_normal(x.shape)) for x in xs]
    out = split(P.hvp(packed(vs, dt)), P.sizes)
    for k, ll in enumerate(prob.lowers):
        ref = ll.hvp(xs[k], th0, vs[k])
        assert rel(out[k], ref) < TOL[precision], (k, rel(out[k], ref))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tv_parity_mask(precision):
    wl = mixed_workload(seed=2, reg="tv")
    P, prob, dt = make(wl, precision, max_recycle=1, max_basis=4)
    rng = np.random.default_rng(2)
    xs = point(wl, rng)
    th0 = np.array([-2.0])
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    g, vals = P.gradient(theta, packed(xs, dt))
    g = split(g, P.sizes)
    for k, ll in enumerate(prob.lowers):
        assert rel(g[k], ll.grad(xs[k], th0)) < TOL[precision]
    P.set_point(theta, packed(xs, dt))
    vs = [r32(rng.standard_normal(x.shape)) for x in xs]
    out = split(P.hvp(packed(vs, dt)), P.sizes)
    for k, ll in enumerate(prob.lowers):
        assert rel(out[k], ll.hvp(xs[k], th0, vs[k])) < TOL[precision]


def test_inpainting_hypergradient_fp32():
    """FP32 Hessian solve and J w at the exact lower-level solution of the inpainting pairs:
    hypergradients within 1e-4 of the checker's.  (phi = s^2 makes the lower level quadratic, so
    x^ = H^{-1} 2 A^T y exactly; with 70 % of the pixels unmeasured H is ill-conditioned, and the
    lower solve itself is checked separately through its first-order condition.)"""
    wl = mixed_workload(seed=3, phi="sq")
    P, prob, dt = make(wl, "fp32", max_recycle=8, max_basis=40)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    xr = []
    for k, ll in enumerate(prob.lowers):
        zero = np.zeros((ll.h, ll.w))
        b = 2.0 * ll.At(ll.y).reshape(-1)
        xv, _, _ = cg(prob.apply_H(k, zero, th), b, np.zeros_like(b), 1e-13 * np.linalg.norm(b), 20000)
        xr.append(r32(xv.reshape(ll.h, ll.w)))
    P.set_point(theta, packed(xr, dt))
    w = P.zeros()
    P.hessian_solve(w, recycle=False, tol=1e-7, relative=True, maxit=4000)
    hg = P.hypergrad(w, per_pair=True)[1].cpu().numpy()
    for k, ll in enumerate(prob.lowers):
        ref = prob.Jw(k, xr[k], th, prob.reference_w(k, xr[k], th))
        assert rel(hg[k], ref) < 1e-4, (k, rel(hg[k], ref))
    # the GPU lower solve reaches its relative gradient tolerance (checked with the checker's gradient)
    x = P.zeros()
    info = P.lower_solve(theta, x, gtol=1e-5, relative=True, max_iters=4000)
    xs = split(x, P.sizes)
    for k, ll in enumerate(prob.lowers):
        g0 = np.linalg.norm(ll.grad(np.zeros_like(xs[k]), th))
        assert np.linalg.norm(ll.grad(xs[k], th)) <= 3e-5 * g0, (k, info[k])
