"""GPU: every entry point called on a pair subset (reordered) gives the full batch's results for
those pairs (per-pair arithmetic is independent; masks, gather and scatter must not change it)."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from tests.gpu_util import DEV, make, packed, r32, rel, split

pytestmark = pytest.mark.gpu
SUB = [2, 0]


def setup():
    wl = synth.uneven_foe([(40, 44), (33, 70), (64, 64)], n_filters=3, f=5, blur_radius=2, seed=21)
    return wl


def test_subset_entry_points_match_full_batch():
    wl = setup()
    P, prob, dt = make(wl, "fp32", max_recycle=6, max_basis=40)
    Q, _, _ = make(wl, "fp32", max_recycle=6, max_basis=40)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    sizes_sub = [P.sizes[k] for k in SUB]
    xf = P.zeros()
    inf_f = P.lower_solve(theta, xf, gtol=1e-5)
    xs = Q.zeros(pairs=SUB)
    inf_s = Q.lower_solve(theta, xs, pairs=SUB, gtol=1e-5)
    XF, XS = split(xf, P.sizes), split(xs, sizes_sub)
    for i, k in enumerate(SUB):
        assert abs(inf_f[k]["iters"] - inf_s[i]["iters"]) <= 1
        assert rel(XS[i], XF[k]) < 1e-5
    # the rest at the full batch's point
    Q.set_point(theta, xf)
    rng = np.random.default_rng(3)
    vs = [r32(rng.standard_normal(s)) for s in P.sizes]
    hf = split(P.hvp(packed(vs, dt)), P.sizes)
    hs = split(Q.hvp(packed([vs[k] for k in SUB], dt), pairs=SUB), sizes_sub)
    for i, k in enumerate(SUB):
        assert rel(hs[i], hf[k]) < 1e-6
    wf = P.zeros()
    P.hessian_solve(wf, recycle=False, tol=1e-6, store_basis=True)
    ws = Q.zeros(pairs=SUB)
    Q.hessian_solve(ws, pairs=SUB, recycle=False, tol=1e-6, store_basis=True)
    WF, WS = split(wf, P.sizes), split(ws, sizes_sub)
    for i, k in enumerate(SUB):
        assert rel(WS[i], WF[k]) < 1e-5
    _, gf = P.hypergrad(wf, per_pair=True)
    _, gs = Q.hypergrad(ws, pairs=SUB, per_pair=True)
    for i, k in enumerate(SUB):
        assert rel(gs[i].cpu().numpy(), gf[k].cpu().numpy()) < 1e-4


def test_subset_refresh_and_recycled_solve_match_full_batch():
    wl = setup()
    P, prob, dt = make(wl, "fp32", max_recycle=6, max_basis=40)
    Q, _, _ = make(wl, "fp32", max_recycle=6, max_basis=40)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    x = P.zeros()
    P.lower_solve(theta, x, gtol=1e-5)
    Q.set_point(theta, x)
    sizes_sub = [P.sizes[k] for k in SUB]
    wf = P.zeros()
    P.hessian_solve(wf, recycle=False, tol=1e-6, store_basis=True)
    ws = Q.zeros(pairs=SUB)
    Q.hessian_solve(ws, pairs=SUB, recycle=False, tol=1e-6, store_basis=True)
    P.ritz_update("RGen-L(R)", 6)
    Q.ritz_update("RGen-L(R)", 6, pairs=SUB)
    for k in SUB:
        assert Q.recycle_dim(k) == P.recycle_dim(k) == 6
    assert Q.recycle_dim(1) == 0
    wf2 = P.zeros()
    inf_f = P.hessian_solve(wf2, recycle=True, tol=1e-6, warm_start=False)
    ws2 = Q.zeros(pairs=SUB)
    inf_s = Q.hessian_solve(ws2, pairs=SUB, recycle=True, tol=1e-6, warm_start=False)
    WF, WS = split(wf2, P.sizes), split(ws2, sizes_sub)
    for i, k in enumerate(SUB):
        assert abs(inf_f[k]["iters"] - inf_s[i]["iters"]) <= 1
        assert rel(WS[i], WF[k]) < 1e-5
