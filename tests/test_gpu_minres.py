"""GPU parity of (recycled) MINRES, Algorithm 3 with the recurrences of Appendix A, against the
FP64 checker: plain MINRES on SPD and on indefinite Hessians (the non-convex phi = log(1 + s^2)
of Section 5.2), a recycled sequence with Ritz-GSV refreshes, the hypergradient-error rule, the
FP32 hypergradient bar, and the graph loop against the host-polled loop."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from oracle import recycle as orc
from oracle.krylov import rminres
from tests.gpu_util import DEV, make, packed, r32, rel, split

pytestmark = pytest.mark.gpu


def small_wl(sizes=((48, 52), (33, 70)), N=3, f=5, rb=2, seed=1):
    return synth.uneven_foe(list(sizes), n_filters=N, f=f, blur_radius=rb, seed=seed)


def indefinite_setup(precision="fp64"):
    """FoE with phi = log(1 + s^2), large filters and weights: phi'' < 0 wherever |K_j x| > 1, and
    the Hessian at a perturbed image has negative eigenvalues (checked on the dense matrix)."""
    wl = small_wl(sizes=((16, 18), (12, 15)), seed=31)
    wl.phi = "log1p"
    P, prob, dt = make(wl, precision)
    th = wl.theta0.copy()
    F = wl.filter_size ** 2 + 1
    for j in range(wl.n_filters):
        th[j * F] = 1.0
        th[j * F + 1:(j + 1) * F] *= 8.0
    if precision == "fp32":
        th = r32(th)
    xs = [wl.x_star[k] + 0.1 * np.random.default_rng(k).standard_normal(wl.x_star[k].shape)
          for k in range(len(wl.pairs))]
    if precision == "fp32":
        xs = [r32(x) for x in xs]
    return wl, P, prob, dt, th, xs


def test_minres_plain_matches_checker_fp64():
    wl = small_wl()
    P, prob, dt = make(wl, "fp64", max_recycle=4, max_basis=60)
    th = wl.theta0
    xs, _ = prob.solve_lower(th, gtol=1e-8)
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w = P.zeros()
    info = P.hessian_solve(w, recycle=False, tol=1e-8, relative=True, maxit=3000, method="minres", warm_start=False)
    ws = split(w, P.sizes)
    for k in range(P.K):
        g = prob.rhs(k, xs[k])
        out = rminres(prob.apply_H(k, xs[k], th), g, np.zeros_like(g), None, None, tol=1e-8 * np.linalg.norm(g),
                      maxit=3000)
        assert abs(info[k]["iters"] - out["iters"]) <= 1, (k, info[k]["iters"], out["iters"])
        assert rel(ws[k], out["w"]) < 1e-8
        # |zeta_k| is the residual norm of MINRES: below the bound for both.  Lanczos without
        # reorthogonalisation amplifies rounding in the final residual: two checker runs that differ
        # only in the summation order of H v (stencils vs the dense matrix) end 2-5 % apart at the
        # same step with iterates equal to 2e-9, so equal steps are compared within 10 %.
        assert info[k]["resid"] < 1e-8 * np.linalg.norm(g) and out["resid"] < 1e-8 * np.linalg.norm(g)
        if info[k]["iters"] == out["iters"]:
            assert abs(info[k]["resid"] - out["resid"]) <= 0.1 * out["resid"]


def test_minres_indefinite_log_phi_fp64():
    wl, P, prob, dt, th, xs = indefinite_setup("fp64")
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w = P.zeros()
    info = P.hessian_solve(w, recycle=False, tol=1e-10, relative=True, maxit=3000, method="minres",
                           warm_start=False)
    ws = split(w, P.sizes)
    for k, ll in enumerate(prob.lowers):
        H = ll.dense_hessian(xs[k], th)
        assert np.linalg.eigvalsh(H)[0] < 0          # indefinite: CG's assumptions fail here
        g = prob.rhs(k, xs[k])
        out = rminres(prob.apply_H(k, xs[k], th), g, np.zeros_like(g), None, None,
                      tol=1e-10 * np.linalg.norm(g), maxit=3000)
        assert abs(info[k]["iters"] - out["iters"]) <= 1, (k, info[k]["iters"], out["iters"])
        assert info[k]["status"] == 0
        wd = np.linalg.solve(H, g.ravel())
        assert rel(ws[k], wd) < 1e-8
        assert rel(ws[k], out["w"]) < 1e-8


def test_rminres_sequence_fp64_matches_checker():
    """Three systems along a theta path with RGen-L(R) refreshes from the Lanczos bases: the GPU's
    recycled MINRES follows the checker's iteration counts (+-1) and solutions."""
    wl = small_wl(sizes=((40, 44),), N=3, seed=4)
    kmax = 60
    P, prob, dt = make(wl, "fp64", max_recycle=6, max_basis=kmax)
    th = wl.theta0.copy()
    rng = np.random.default_rng(0)
    U = C = None
    V = None
    w_prev = None
    for i in range(3):
        xs, _ = prob.solve_lower(th, gtol=1e-8)
        x = xs[0]
        P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
        AH = prob.apply_H(0, x, th)
        if V is not None:
            P.ritz_update("RGen-L(R)", 6)
            Up = U if U is not None else np.zeros((x.size, 0))
            U, C, Z, _ = orc.refresh(Up, V, AH, lambda v: prob.Jw(0, x, th, v.reshape(x.shape)), 6, "rgsv", "L", "R")
            assert P.recycle_dim(0) == U.shape[1]
        g = prob.rhs(0, x)
        w0 = np.zeros_like(g) if w_prev is None else w_prev
        out = rminres(AH, g, w0, U, C, tol=1e-7 * np.linalg.norm(g), maxit=2000)
        wg = packed([w0.reshape(x.shape)], dt)
        info = P.hessian_solve(wg, recycle=True, tol=1e-7, relative=True, warm_start=True, maxit=2000,
                               method="minres")
        assert abs(info[0]["iters"] - out["iters"]) <= 1, (i, info[0]["iters"], out["iters"])
        assert rel(wg.cpu().numpy(), out["w"]) < 1e-7
        # the library keeps the most recent `kmax` Lanczos vectors
        V = out["V"][:, -kmax:]
        w_prev = out["w"]
        th = th - 0.005 * rng.standard_normal(th.shape)


def test_rminres_nsc_fp64():
    """RGen-L(R)-NSC with recycled MINRES: the estimate ||Z^T res|| follows the explicit-residual
    recurrence of Appendix A; the GPU stops within 10 % (at least two) of the checker's iterations
    (the spread the choice of orthonormal basis of range(W) causes, as for CG) below the threshold."""
    wl = small_wl(sizes=((40, 44),), N=3, seed=4)
    kmax = 60
    P, prob, dt = make(wl, "fp64", max_recycle=6, max_basis=kmax)
    th = wl.theta0.copy()
    rng = np.random.default_rng(3)
    U = C = Z = V = None
    w_prev = None
    tol, scale = 1e-6, 2.5
    for i in range(3):
        xs, _ = prob.solve_lower(th, gtol=1e-7)
        x = xs[0]
        P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
        AH = prob.apply_H(0, x, th)
        if V is not None:
            P.ritz_update("RGen-L(R)", 6)
            Up = U if U is not None else np.zeros((x.size, 0))
            U, C, Z, _ = orc.refresh(Up, V, AH, lambda v: prob.Jw(0, x, th, v.reshape(x.shape)), 6, "rgsv", "L", "R")
        g = prob.rhs(0, x)
        w0 = np.zeros_like(g) if w_prev is None else w_prev
        if Z is None:
            out = rminres(AH, g, w0, U, C, tol=tol * np.linalg.norm(g), maxit=2000)
        else:
            out = rminres(AH, g, w0, U, C, tol=tol * scale, maxit=2000, stop="nsc", Z=Z)
        wg = packed([w0.reshape(x.shape)], dt)
        info = P.hessian_solve(wg, recycle=True, nsc=True, tol=tol, relative=True, warm_start=True, maxit=2000,
                               nsc_scale=[scale], method="minres")
        bar = 1 if Z is None else max(2, out["iters"] // 10)
        assert abs(info[0]["iters"] - out["iters"]) <= bar, (i, info[0]["iters"], out["iters"])
        if Z is not None:
            assert info[0]["nsc"] < tol * scale and out["nsc"] < tol * scale
        assert rel(wg.cpu().numpy(), out["w"]) < (1e-7 if Z is None else 1e-5)
        V, w_prev = out["V"][:, -kmax:], out["w"]
        th = th - 0.005 * rng.standard_normal(th.shape)


def test_minres_hypergradient_fp32():
    """FP32 MINRES (plain and on an indefinite Hessian): hypergradients within the 1e-4 bar of the
    checker's dense-solve reference."""
    wl = small_wl(sizes=((56, 56), (40, 72)), N=4, seed=11)
    P, prob, dt = make(wl, "fp32", max_recycle=8, max_basis=60)
    th = r32(wl.theta0)
    xs = [r32(x) for x in prob.solve_lower(th, gtol=1e-8)[0]]
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w = P.zeros()
    P.hessian_solve(w, recycle=False, tol=1e-6, relative=True, maxit=3000, method="minres", warm_start=False)
    hg = P.hypergrad(w, per_pair=True)[1].cpu().numpy()
    for k in range(P.K):
        wref = prob.reference_w(k, xs[k], th)
        assert rel(hg[k], prob.Jw(k, xs[k], th, wref)) < 1e-4

    wl2, P2, prob2, dt2, th2, xs2 = indefinite_setup("fp32")
    P2.set_point(torch.tensor(th2, dtype=torch.float64, device=DEV), packed(xs2, dt2))
    w2 = P2.zeros()
    P2.hessian_solve(w2, recycle=False, tol=1e-6, relative=True, maxit=3000, method="minres", warm_start=False)
    hg2 = P2.hypergrad(w2, per_pair=True)[1].cpu().numpy()
    for k, ll in enumerate(prob2.lowers):
        H = ll.dense_hessian(xs2[k], th2)
        wd = np.linalg.solve(H, prob2.rhs(k, xs2[k]).ravel()).reshape(xs2[k].shape)
        assert rel(hg2[k], prob2.Jw(k, xs2[k], th2, wd)) < 1e-4


def test_minres_graph_matches_stream_loop():
    """The MINRES loop as one CUDA-graph launch gives the host-polled loop's iterations and
    bit-identical solutions."""
    wl = small_wl(sizes=((64, 70), (33, 40), (90, 31)), N=3, seed=17)
    P, prob, dt = make(wl, "fp32", max_recycle=6, max_basis=40)
    th = r32(wl.theta0)
    xs = [r32(x + 0.01) for x in wl.x_star]
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w0 = P.zeros()
    P.hessian_solve(w0, recycle=False, tol=1e-4, store_basis=True, graph=False, method="minres")
    P.ritz_update("RGen-L(R)", 6)
    outs = []
    for graph in (False, True, True):
        w = P.zeros()
        info = P.hessian_solve(w, recycle=True, tol=1e-6, store_basis=False, graph=graph, method="minres")
        assert P.graph_used() == graph
        outs.append(([d["iters"] for d in info], w.cpu().numpy()))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[1][1], outs[2][1])
