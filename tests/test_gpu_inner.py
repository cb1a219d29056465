"""GPU parity of the inner recycle refresh (eq. (3.4)): the projected problem is built with the
Hessian of the last solve, rebuilt on the GPU from that CG solve's Lanczos record (no Hessian
actions), and the selected space is paired with C = H U at the new point.  The checker projects
with explicit Hessian actions of the old operator (oracle.recycle.refresh_inner)."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from oracle import recycle as orc
from oracle.krylov import rcg
from tests.gpu_util import DEV, make, packed, r32, rel

pytestmark = pytest.mark.gpu


def exported(P, k, dtype):
    blob = P.recycle_export(k)
    s = P.recycle_dim(k)
    h, w = P.sizes[k]
    n = h * w
    esz = np.dtype(dtype).itemsize
    arr = np.frombuffer(blob[32:32 + 2 * s * n * esz], dtype=dtype).astype(np.float64)
    return arr[:s * n].reshape(s, n).T, arr[s * n:2 * s * n].reshape(s, n).T


def min_cos(A, B):
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return np.linalg.svd(Qa.T @ Qb, compute_uv=False).min()


@pytest.mark.parametrize("kind", ["Ritz-S", "RGen-L(R)"])
def test_inner_refresh_matches_checker_fp64(kind):
    """Two refreshes along a theta path (the second with a non-empty previous recycle space, so the
    C^T H p_j part of the relation is exercised): the GPU's inner space equals the checker's."""
    wl = synth.uneven_foe([(40, 44)], n_filters=3, f=5, blur_radius=2, seed=4)
    kmax, s = 40, 6
    P, prob, dt = make(wl, "fp64", max_recycle=s, max_basis=kmax)
    st = {"Ritz-S": ("ritz", "S", "R"), "RGen-L(R)": ("rgsv", "L", "R")}[kind]
    rng = np.random.default_rng(5)
    th = wl.theta0.copy()
    U = C = None
    w_prev = None
    AH_old = None
    V = None
    for i in range(3):
        xs, _ = prob.solve_lower(th, gtol=1e-8)
        x = xs[0]
        P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
        AH = prob.apply_H(0, x, th)
        if V is not None:
            P.ritz_update(kind, s, variant="inner")
            Up = U if U is not None else np.zeros((x.size, 0))
            U, C, _, _ = orc.refresh_inner(Up, V, AH_old, AH, lambda v: prob.Jw(0, x, th, v.reshape(x.shape)),
                                          s, *st)
            Ug, Cg = exported(P, 0, np.float64)
            assert Ug.shape == U.shape
            assert min_cos(Ug, U) > 1 - 1e-8, (i, min_cos(Ug, U))
            HU = np.stack([AH(Ug[:, j]) for j in range(s)], 1)
            assert rel(HU, Cg) < 1e-9
            np.testing.assert_allclose(Cg.T @ Cg, np.eye(s), atol=1e-10)
        g = prob.rhs(0, x)
        w0 = np.zeros_like(g) if w_prev is None else w_prev
        out = rcg(AH, g, w0, U, C, tol=1e-7 * np.linalg.norm(g), maxit=2000)
        wg = packed([w0.reshape(x.shape)], dt)
        info = P.hessian_solve(wg, recycle=True, tol=1e-7, relative=True, warm_start=True, maxit=2000,
                               store_basis="lanczos")
        assert abs(info[0]["iters"] - out["iters"]) <= 1, (i, info[0]["iters"], out["iters"])
        assert rel(wg.cpu().numpy(), out["w"]) < 1e-7
        # the record keeps the first kmax residuals: v_0 .. v_{m-1} span the basis, m = min(iters, kmax - 1)
        m = min(info[0]["iters"], kmax - 1)
        assert P.basis_size(0) == m
        V = out["V"][:, :m]
        AH_old = AH
        w_prev = out["w"]
        th = th - 0.005 * rng.standard_normal(th.shape)


def test_inner_refresh_invariants_fp32():
    """FP32 inner refresh for every vector type: C = H U at the new point and C^T C = I."""
    wl = synth.uneven_foe([(64, 64), (37, 45)], n_filters=4, f=5, blur_radius=2, seed=7)
    P, prob, dt = make(wl, "fp32", max_recycle=8, max_basis=40)
    th = r32(wl.theta0)
    xs = [r32(x) for x in prob.solve_lower(th, gtol=1e-8)[0]]
    rng = np.random.default_rng(2)
    for kind in ["Ritz-S", "RGen-L(R)", "HRitz-L"]:
        P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
        w = P.zeros()
        P.hessian_solve(w, recycle=False, tol=1e-5, store_basis="lanczos")
        th2 = r32(th - 0.01 * rng.standard_normal(th.shape))
        xs2 = [r32(x + 0.01 * rng.standard_normal(x.shape)) for x in xs]
        P.set_point(torch.tensor(th2, dtype=torch.float64, device=DEV), packed(xs2, dt))
        P.ritz_update(kind, 8, variant="inner")
        for k in range(P.K):
            assert P.recycle_dim(k) == 8
            Ug, Cg = exported(P, k, np.float32)
            h, wd = P.sizes[k]
            np.testing.assert_allclose(Cg.T @ Cg, np.eye(8), atol=2e-4)
            HU = np.stack([prob.lowers[k].hvp(xs2[k], th2, Ug[:, j].reshape(h, wd)).ravel() for j in range(8)], 1)
            assert np.linalg.norm(HU - Cg) / np.linalg.norm(Cg) < 1e-3, kind


def test_inner_refresh_needs_a_lanczos_record():
    wl = synth.uneven_foe([(30, 31)], n_filters=2, f=3, blur_radius=1, seed=3)
    P, prob, dt = make(wl, "fp32", max_recycle=4, max_basis=20)
    th = r32(wl.theta0)
    xs = [r32(x + 0.05 * np.random.default_rng(1).standard_normal(x.shape)) for x in wl.x_star]
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w = P.zeros()
    P.hessian_solve(w, recycle=False, tol=1e-4, store_basis=True)
    with pytest.raises(Exception, match="Lanczos record"):
        P.ritz_update("Ritz-S", 4, variant="inner")
    with pytest.raises(Exception, match="MINRES keeps"):
        P.hessian_solve(w, recycle=False, tol=1e-4, store_basis="lanczos", method="minres")


def test_inner_refresh_leaves_only_a_zero_step_pair_without_space():
    """A pair whose recorded solve ran without its recycle space and took no step (warm start already
    at the solution) has nothing relating its space to the new Hessian: the inner refresh clears
    that pair alone (BL_EBREAKDOWN, reported by the binding as False) and refreshes the others as
    the checker does."""
    wl = synth.uneven_foe([(40, 44), (36, 30)], n_filters=3, f=5, blur_radius=2, seed=9)
    kmax, s = 40, 4
    P, prob, dt = make(wl, "fp64", max_recycle=s, max_basis=kmax)
    rng = np.random.default_rng(9)
    th = wl.theta0.copy()
    ths = [th, th - 0.005 * rng.standard_normal(th.shape)]
    ths.append(ths[1] - 0.005 * rng.standard_normal(th.shape))
    # points to a gradient of 1e-8 (any fixed points serve: both sides evaluate H and J there); 1e-9
    # sits near the FP64 line search's rounding floor on some hosts, where these solves take minutes
    pts = [prob.solve_lower(t, gtol=1e-8)[0] for t in ths]
    # step 0: plain solves with the Lanczos record; refresh at the next point gives both pairs a space
    P.set_point(torch.tensor(ths[0], dtype=torch.float64, device=DEV), packed(pts[0], dt))
    w = P.zeros()
    P.hessian_solve(w, recycle=True, tol=1e-7, relative=True, warm_start=False, maxit=2000, store_basis="lanczos")
    P.set_point(torch.tensor(ths[1], dtype=torch.float64, device=DEV), packed(pts[1], dt))
    assert P.ritz_update("Ritz-S", s, variant="inner")
    assert P.recycle_dim(0) == s and P.recycle_dim(1) == s
    # step 1: pair 0 starts at its exact solution (no step), pair 1 from zero; no recycling
    x1 = pts[1]
    wstar0 = prob.reference_w(0, x1[0], ths[1])
    w = packed([wstar0.reshape(x1[0].shape), np.zeros(x1[1].shape)], dt)
    info = P.hessian_solve(w, recycle=False, tol=1e-7, relative=True, warm_start=True, maxit=2000,
                           store_basis="lanczos")
    assert info[0]["iters"] == 0 and info[1]["iters"] > 0
    AH1 = prob.apply_H(1, x1[1], ths[1])
    g1 = prob.rhs(1, x1[1])
    out = rcg(AH1, g1, np.zeros_like(g1), None, None, tol=1e-7 * np.linalg.norm(g1), maxit=2000)
    assert abs(info[1]["iters"] - out["iters"]) <= 1
    m = min(info[1]["iters"], kmax - 1)
    V1 = out["V"][:, :m]
    # step 2: inner refresh
    x2 = pts[2]
    P.set_point(torch.tensor(ths[2], dtype=torch.float64, device=DEV), packed(x2, dt))
    assert P.ritz_update("Ritz-S", s, variant="inner") is False
    assert P.recycle_dim(0) == 0
    assert P.recycle_dim(1) == s
    AH2 = prob.apply_H(1, x2[1], ths[2])
    U, C, _, _ = orc.refresh_inner(np.zeros((x2[1].size, 0)), V1, AH1, AH2,
                                   lambda v: prob.Jw(1, x2[1], ths[2], v.reshape(x2[1].shape)), s, "ritz", "S", "R")
    Ug, Cg = exported(P, 1, np.float64)
    assert min_cos(Ug, U) > 1 - 1e-8, min_cos(Ug, U)
    # the cleared pair solves as plain CG next, the refreshed one with its new space
    w = P.zeros()
    info = P.hessian_solve(w, recycle=True, tol=1e-7, relative=True, warm_start=False, maxit=2000)
    g0 = prob.rhs(0, x2[0])
    ref0 = rcg(prob.apply_H(0, x2[0], ths[2]), g0, np.zeros_like(g0), None, None, tol=1e-7 * np.linalg.norm(g0),
               maxit=2000)
    assert abs(info[0]["iters"] - ref0["iters"]) <= 1
