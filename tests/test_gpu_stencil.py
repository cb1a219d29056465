"""GPU parity of the stencil entry points (bl_forward, bl_gradient, bl_hvp, bl_hypergrad's J w)
against the FP64 checker, element by element, on seeded inputs spanning several tiles with
ragged tails.  Tolerances: 1e-5 relative (FP32 Hessian action, the stated bar), 1e-12 (FP64)."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from oracle import operators as ops
from tests.gpu_util import DEV, make, max_elem, packed, r32, rel, split

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}

CASES = [
    # (sizes, n_filters, f, blur_radius)
    ([(70, 131)], 3, 5, 2),
    ([(37, 45), (130, 64), (1, 9), (9, 1)], 4, 3, 4),
    ([(61, 77), (128, 128)], 2, 7, 1),
    ([(64, 64)], 2, 1, 3),
]


def workload(sizes, N, f, rb, seed=0):
    wl = synth.uneven_foe(sizes, n_filters=N, f=f, blur_radius=rb, seed=seed)
    # theta with non-trivial weights so every term matters
    return wl


def point(prob, wl, rng):
    return [r32(np.clip(x + 0.05 * rng.standard_normal(x.shape), -0.2, 1.2)) for x in wl.x_star]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_forward_blur(case, precision):
    sizes, N, f, rb = CASES[case]
    wl = workload(sizes, N, f, rb)
    P, prob, dt = make(wl, precision)
    out = P.forward(packed(prob.x_star, dt))
    for got, xs, ll in zip(split(out, P.sizes), prob.x_star, prob.lowers):
        assert rel(got, ops.blur(xs, ll.G)) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_hvp_parity(case, precision):
    sizes, N, f, rb = CASES[case]
    wl = workload(sizes, N, f, rb, seed=case)
    P, prob, dt = make(wl, precision)
    rng = np.random.default_rng(case)
    xs = point(prob, wl, rng)
    th0 = r32(wl.theta0) if precision == "fp32" else wl.theta0
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    vs = [r32(rng.standard_normal(x.shape)) for x in xs]
    out = split(P.hvp(packed(vs, dt)), P.sizes)
    for k, ll in enumerate(prob.lowers):
        ref = ll.hvp(xs[k], th0, vs[k])
        assert rel(out[k], ref) < TOL[precision], (k, rel(out[k], ref))
        assert max_elem(out[k], ref) < TOL[precision], (k, max_elem(out[k], ref))


# Every width a multiple of 4: the FP32 Hessian action runs the TMA-staged kernel.  Several tiles,
# ragged tails in both directions, images narrower and shorter than one tile, every blur radius.
TMA_CASES = [
    # (sizes, n_filters, f, blur_radius)
    ([(70, 132), (37, 44), (9, 4)], 3, 5, 2),
    ([(128, 192), (67, 60)], 16, 5, 4),
    ([(61, 76), (130, 64)], 2, 7, 3),
    ([(64, 64), (5, 8)], 2, 1, 4),
    ([(45, 124)], 4, 3, 1),
    ([(33, 68), (120, 4)], 2, 5, 0),
]


@pytest.mark.parametrize("case", range(len(TMA_CASES)))
def test_hvp_parity_tma_path(case):
    """The TMA-staged FP32 Hessian action against the checker, per element (tile seams, image borders,
    the zero-filled halo of the tensor copies) and in norm."""
    sizes, N, f, rb = TMA_CASES[case]
    wl = workload(sizes, N, f, rb, seed=40 + case)
    P, prob, dt = make(wl, "fp32")
    assert P.hvp_tma()
    rng = np.random.default_rng(40 + case)
    xs = point(prob, wl, rng)
    th0 = r32(wl.theta0)
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    for rep in range(2):
        vs = [r32(rng.standard_normal(x.shape)) for x in xs]
        out = split(P.hvp(packed(vs, dt)), P.sizes)
        for k, ll in enumerate(prob.lowers):
            ref = ll.hvp(xs[k], th0, vs[k])
            assert rel(out[k], ref) < TOL["fp32"], (k, rel(out[k], ref))
            assert max_elem(out[k], ref) < TOL["fp32"], (k, max_elem(out[k], ref))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_gradient_and_value_parity(case, precision):
    sizes, N, f, rb = CASES[case]
    wl = workload(sizes, N, f, rb, seed=10 + case)
    P, prob, dt = make(wl, precision)
    rng = np.random.default_rng(10 + case)
    xs = point(prob, wl, rng)
    th0 = r32(wl.theta0) if precision == "fp32" else wl.theta0
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    g, vals = P.gradient(theta, packed(xs, dt))
    g = split(g, P.sizes)
    vals = vals.cpu().numpy()
    for k, ll in enumerate(prob.lowers):
        assert rel(g[k], ll.grad(xs[k], th0)) < TOL[precision]
        assert abs(vals[k] - ll.value(xs[k], th0)) < TOL[precision] * abs(ll.value(xs[k], th0))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_jw_parity(case, precision):
    sizes, N, f, rb = CASES[case]
    wl = workload(sizes, N, f, rb, seed=20 + case)
    P, prob, dt = make(wl, precision)
    rng = np.random.default_rng(20 + case)
    xs = point(prob, wl, rng)
    th0 = r32(wl.theta0) if precision == "fp32" else wl.theta0
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    ws = [r32(rng.standard_normal(x.shape)) for x in xs]
    mean, per = P.hypergrad(packed(ws, dt), per_pair=True)
    per = per.cpu().numpy()
    refs = [ll.Jw(xs[k], th0, ws[k]) for k, ll in enumerate(prob.lowers)]
    for k in range(len(refs)):
        # FP32 inputs: J w sums n products; compare per component against the scale of the vector
        assert rel(per[k], refs[k]) < (1e-5 if precision == "fp32" else 1e-11), (k, rel(per[k], refs[k]))
    assert rel(mean.cpu().numpy(), np.mean(refs, axis=0)) < (1e-5 if precision == "fp32" else 1e-11)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tv_parity(precision):
    wl = synth.tv_32()
    wl.pairs = wl.pairs + [synth.PairSpec(13, 21, 1.2, 1, 0.01)]
    rng = np.random.default_rng(5)
    wl.x_star = wl.x_star + [rng.uniform(0, 1, (13, 21))]
    wl.noise = wl.noise + [0.01 * rng.standard_normal((13, 21))]
    P, prob, dt = make(wl, precision, max_recycle=1, max_basis=4)
    xs = [r32(x + 0.05 * rng.standard_normal(x.shape)) for x in wl.x_star]
    th = np.array([-2.5])
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    vs = [r32(rng.standard_normal(x.shape)) for x in xs]
    hv = split(P.hvp(packed(vs, dt)), P.sizes)
    g, vals = P.gradient(theta, packed(xs, dt))
    g = split(g, P.sizes)
    P.set_point(theta, packed(xs, dt))
    mean, per = P.hypergrad(packed(vs, dt), per_pair=True)
    tol = 1e-5 if precision == "fp32" else 1e-12
    for k, ll in enumerate(prob.lowers):
        assert rel(hv[k], ll.hvp(xs[k], th, vs[k])) < tol
        assert rel(g[k], ll.grad(xs[k], th)) < tol
        assert rel(per[k].cpu().numpy(), ll.Jw(xs[k], th, vs[k])) < tol * 10
        assert abs(vals[k].item() - ll.value(xs[k], th)) < tol * ll.value(xs[k], th)
