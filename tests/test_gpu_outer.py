"""GPU parity of the outer machinery: the hypergradient-error stopping rule (Section 4), gradient
descent with backtracking (Algorithms 1-2) on the TV workload, the autograd Function (its backward
is the recycled solve + J w) against the checker and against finite differences, and recycle-space
checkpointing."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from paper_2412_08264_gb300.autograd import lower_level_solve
from paper_2412_08264_gb300.outer import Engine, gradient_descent
from oracle import recycle as orc
from oracle.bilevel import gradient_descent as oracle_gd
from oracle.krylov import rcg
from tests.gpu_util import DEV, make, packed, rel, split

pytestmark = pytest.mark.gpu


def test_nsc_stopping_matches_checker_fp64():
    """RGen-L(R)-NSC on a three-system sequence: the GPU stops on ||Z^T r|| < tol * scale within
    10 % (at least two) of the checker's iterations; the first system (no Ritz-GSV space yet) uses
    the residual rule and matches within one.  The Ritz-GSV selection passes through T^{-1} (condition ~1e7 here),
    so FP64 rounding in the choice of orthonormal basis of range(W) -- which the method leaves
    open -- moves the NSC stop by up to two iterations and its final estimate by ~15 %: the
    checker itself shows this spread between an SVD, a pivoted-Cholesky and an eigenvector basis."""
    wl = synth.uneven_foe([(40, 44)], n_filters=3, f=5, blur_radius=2, seed=4)
    P, prob, dt = make(wl, "fp64", max_recycle=6, max_basis=60)
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
            out = rcg(AH, g, w0, U, C, tol=tol * np.linalg.norm(g), maxit=2000, kmax_store=60)
        else:
            out = rcg(AH, g, w0, U, C, tol=tol * scale, maxit=2000, stop="nsc", Z=Z, kmax_store=60)
        wg = packed([w0.reshape(x.shape)], dt)
        info = P.hessian_solve(wg, recycle=True, nsc=True, tol=tol, relative=True, warm_start=True, maxit=2000,
                               nsc_scale=[scale])
        bar = 1 if Z is None else max(2, out["iters"] // 10)
        assert abs(info[0]["iters"] - out["iters"]) <= bar, (i, info[0]["iters"], out["iters"])
        if Z is not None:
            # both stopped below the threshold; at the same stopping step the estimates agree within
            # the spread of the basis choice (a one- or two-step shift changes them by whole steps)
            assert info[0]["nsc"] < tol * scale and out["nsc"] < tol * scale
            if info[0]["iters"] == out["iters"]:
                assert abs(info[0]["nsc"] - out["nsc"]) <= 0.25 * tol * scale
        assert rel(wg.cpu().numpy(), out["w"]) < (1e-7 if Z is None else 1e-5)
        V, w_prev = out["V"], out["w"]
        th = th - 0.005 * rng.standard_normal(th.shape)


def test_gradient_descent_tv_matches_checker_fp64():
    """Algorithms 1-2 on the 32x32 TV workload (FP64): the GPU engine and the checker follow the same
    theta trajectory for three outer steps."""
    wl = synth.tv_32()
    P, prob, dt = make(wl, "fp64", max_recycle=1, max_basis=8)
    gtol = 1e-10
    eng = Engine(P, strategy="none", rtol=1e-10, lower_gtol=gtol, lower_relative=False, lower_max_iters=20000,
                 maxit=20000)
    th_gpu, hist = gradient_descent(eng, wl.theta0, 3)

    def solve(k, xh, th, g):
        return prob.reference_w(k, xh, th)

    th_cpu, _, thetas = oracle_gd(prob, wl.theta0, 3, solve, gtol_lower=gtol)
    assert abs(th_gpu[0] - th_cpu[0]) < 1e-7 * max(1.0, abs(th_cpu[0])), (th_gpu, th_cpu)
    assert hist[-1].loss < hist[0].loss


def test_autograd_backward_matches_checker_and_fd_fp64():
    wl = synth.uneven_foe([(24, 27), (20, 31)], n_filters=3, f=5, blur_radius=2, seed=12)
    wl.theta0[0::26] = -1.5          # stronger regularisation: faster, better conditioned lower solves
    P, prob, dt = make(wl, "fp64", max_recycle=4, max_basis=40)
    eng = Engine(P, strategy="RGen-L(R)", s=4, rtol=1e-12, lower_gtol=1e-9, lower_max_iters=5000, maxit=5000)
    xstar = packed(prob.x_star, dt)
    theta = torch.tensor(wl.theta0, dtype=torch.float64, device=DEV, requires_grad=True)

    def loss_of(th):
        x = lower_level_solve(th, eng)
        return 0.5 * ((x - xstar) ** 2).sum() / P.K

    L = loss_of(theta)
    L.backward()
    grad = theta.grad.cpu().numpy()
    # checker: the same hypergradient from its own lower solve and dense reference solve
    # (5e-9: FP64 Armijo steps stop resolving decreases of Phi just above 1e-9 on this problem)
    xs, _ = prob.solve_lower(wl.theta0, gtol=5e-9)
    ws = [prob.reference_w(k, xs[k], wl.theta0) for k in range(P.K)]
    ref = prob.hypergradient(wl.theta0, xs, ws)
    assert rel(grad, ref) < 1e-6, rel(grad, ref)
    # central finite differences of L along random directions (lower solves on the GPU, FP64)
    rng = np.random.default_rng(0)
    # central differences through L-BFGS lower solves stopped at a relative gradient of 1e-9: their
    # stopping error enters divided by 2h (noise ~1e-6 at h = 1e-4), while h = 1e-3 already shows
    # O(h^2) truncation of ~1e-4 on this loss, so the difference is held to 1e-4; the backward pass
    # itself is held to 1e-6 against the checker's hypergradient above
    h = 1e-4
    for _ in range(3):
        d = rng.standard_normal(P.p)
        d /= np.linalg.norm(d)
        dd = torch.tensor(d, dtype=torch.float64, device=DEV)
        with torch.no_grad():
            lp = float(loss_of(theta.detach() + h * dd))
            lm = float(loss_of(theta.detach() - h * dd))
        fd = (lp - lm) / (2 * h)
        an = float(grad @ d)
        assert abs(fd - an) < 1e-4 * max(abs(an), 1e-3 * np.linalg.norm(grad)), (fd, an)


def test_recycle_checkpoint_round_trip():
    """Exporting the recycle state and importing it into a fresh problem reproduces the next solve."""
    wl = synth.uneven_foe([(48, 50), (36, 60)], n_filters=3, f=5, blur_radius=2, seed=21)
    P1, prob, dt = make(wl, "fp32", max_recycle=8, max_basis=40)
    e1 = Engine(P1, strategy="RGen-L(R)", s=8, rtol=1e-5)
    th = wl.theta0.copy()
    for i in range(2):
        e1.loss_and_hypergrad(torch.tensor(th, dtype=torch.float64, device=DEV))
        th = th - 1e-3 * np.sign(np.random.default_rng(i).standard_normal(th.shape))
    sd = e1.state_dict()
    P2, _, _ = make(wl, "fp32", max_recycle=8, max_basis=40, oracle=prob)
    e2 = Engine(P2, strategy="RGen-L(R)", s=8, rtol=1e-5)
    e2.load_state_dict(sd)
    thd = torch.tensor(th, dtype=torch.float64, device=DEV)
    # same point on both; the imported space must give the same recycled solve without a refresh
    x1, _ = e1.lower(thd)
    P2.set_point(thd, x1)
    P1.set_point(thd, x1)
    w1, w2 = e1.w.clone(), e2.w.clone()
    i1 = P1.hessian_solve(w1, recycle=True, tol=1e-5, store_basis=False)
    i2 = P2.hessian_solve(w2, recycle=True, tol=1e-5, store_basis=False)
    assert [a["iters"] for a in i1] == [b["iters"] for b in i2]
    assert [P1.recycle_dim(k) for k in range(2)] == [P2.recycle_dim(k) for k in range(2)] == [8, 8]
    assert rel(w1.cpu().numpy(), w2.cpu().numpy()) < 1e-6
