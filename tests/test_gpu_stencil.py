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


@pytest.mark.parametrize("variant", ["generic", "64"])
@pytest.mark.parametrize("case", range(len(TMA_CASES)))
def test_hvp_parity_tma_path(case, variant):
    """The TMA-staged FP32 Hessian action against the checker, per element (tile seams, image borders,
    the zero-filled halo of the tensor copies) and in norm, for each tile variant: the generic side
    tile_out(f) and, for 3x3 and 5x5 filters, 64 x 64 (forced for every pair)."""
    sizes, N, f, rb = TMA_CASES[case]
    if variant == "64" and f not in (3, 5):
        pytest.skip("the 64 x 64 variant exists for 3x3 and 5x5 filters")
    wl = workload(sizes, N, f, rb, seed=40 + case)
    P, prob, dt = make(wl, "fp32")
    assert P.hvp_tma()
    side = 64 if variant == "64" else {1: 64, 3: 60, 5: 60, 7: 56}[f]
    for k in range(P.K):
        assert P.hvp_tile(k) in ((60, 64) if f in (3, 5) else (side,))
        P.set_hvp_tile(k, side)
        assert P.hvp_tile(k) == side
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


@pytest.mark.parametrize("variant", ["generic", "64"])
@pytest.mark.parametrize("case", range(len(TMA_CASES)))
def test_gradient_and_value_parity_tma_path(case, variant):
    """The TMA-staged gradient of Phi and its value partials against the checker (per element and in
    norm), for each tile variant."""
    sizes, N, f, rb = TMA_CASES[case]
    if variant == "64" and f not in (3, 5):
        pytest.skip("the 64 x 64 variant exists for 3x3 and 5x5 filters")
    wl = workload(sizes, N, f, rb, seed=60 + case)
    P, prob, dt = make(wl, "fp32")
    assert P.hvp_tma()
    side = 64 if variant == "64" else {1: 64, 3: 60, 5: 60, 7: 56}[f]
    for k in range(P.K):
        P.set_hvp_tile(k, side)
    rng = np.random.default_rng(60 + case)
    xs = point(prob, wl, rng)
    th0 = r32(wl.theta0)
    theta = torch.tensor(th0, dtype=torch.float64, device=DEV)
    g, vals = P.gradient(theta, packed(xs, dt))
    g = split(g, P.sizes)
    vals = vals.cpu().numpy()
    for k, ll in enumerate(prob.lowers):
        ref = ll.grad(xs[k], th0)
        assert rel(g[k], ref) < 1e-5, (k, rel(g[k], ref))
        assert max_elem(g[k], ref) < 1e-5, (k, max_elem(g[k], ref))
        assert abs(vals[k] - ll.value(xs[k], th0)) < 1e-5 * abs(ll.value(xs[k], th0))


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


def test_tv_parity_tma_path():
    """FP32 TV problem whose every width is a multiple of 4: the Hessian action runs the TMA-staged TV
    kernel (several tiles, ragged rows, every blur radius); per element and in norm against the
    checker, and through the refresh's multi-column products (C = H U on the exported space)."""
    wl = synth.tv_32()
    rng = np.random.default_rng(6)
    sizes = [(32, 32, 1.5, 2), (70, 132, 2.0, 4), (13, 20, 1.2, 1), (67, 64, 1.0, 0), (9, 8, 1.3, 3)]
    wl.pairs = [synth.PairSpec(h, w, s, r, 0.01) for h, w, s, r in sizes]
    wl.x_star = [rng.uniform(0, 1, (h, w)) for h, w, _, _ in sizes]
    wl.noise = [0.01 * rng.standard_normal((h, w)) for h, w, _, _ in sizes]
    P, prob, dt = make(wl, "fp32", max_recycle=4, max_basis=20)
    assert P.hvp_tma()
    xs = [r32(x + 0.05 * rng.standard_normal(x.shape)) for x in wl.x_star]
    th = np.array([-2.5])
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    for rep in range(2):
        vs = [r32(rng.standard_normal(x.shape)) for x in xs]
        hv = split(P.hvp(packed(vs, dt)), P.sizes)
        for k, ll in enumerate(prob.lowers):
            ref = ll.hvp(xs[k], th, vs[k])
            assert rel(hv[k], ref) < 1e-5, (k, rel(hv[k], ref))
            assert max_elem(hv[k], ref) < 1e-5, (k, max_elem(hv[k], ref))
    w = P.zeros()
    P.hessian_solve(w, recycle=False, tol=1e-5, store_basis=True)
    P.ritz_update("Ritz-S", 4)
    for k in range(P.K):
        s = P.recycle_dim(k)
        blob = P.recycle_export(k)
        h, wd = P.sizes[k]
        n = h * wd
        arr = np.frombuffer(blob[32:32 + 2 * s * n * 4], dtype=np.float32).astype(np.float64)
        U = arr[:s * n].reshape(s, n).T
        Cm = arr[s * n:2 * s * n].reshape(s, n).T
        HU = np.stack([prob.lowers[k].hvp(xs[k], th, U[:, j].reshape(h, wd)).ravel() for j in range(s)], 1)
        assert np.linalg.norm(HU - Cm) / np.linalg.norm(Cm) < 1e-3, k


def test_tile_variants_give_identical_results():
    """Every output pixel of the Hessian action and the gradient is formed by one thread in the same
    order of operations whatever the tile geometry, so the 60 x 60 and 64 x 64 variants agree bit for
    bit (the variant is a speed choice only)."""
    sizes, N, f, rb = TMA_CASES[1]
    wl = workload(sizes, N, f, rb, seed=70)
    P, prob, dt = make(wl, "fp32")
    rng = np.random.default_rng(70)
    xs = point(prob, wl, rng)
    theta = torch.tensor(r32(wl.theta0), dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    v = packed([r32(rng.standard_normal(x.shape)) for x in xs], dt)
    out = {}
    for side in (60, 64):
        for k in range(P.K):
            P.set_hvp_tile(k, side)
        g, vals = P.gradient(theta, packed(xs, dt))
        P.set_point(theta, packed(xs, dt))
        out[side] = (P.hvp(v), g, vals)
    assert torch.equal(out[60][0], out[64][0])
    assert torch.equal(out[60][1], out[64][1])
