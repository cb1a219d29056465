"""GPU parity of the solvers: plain and recycled CG, the recycle refresh, the L-BFGS lower
solve and the full hypergradient, against the FP64 checker on the same inputs.

Bars: FP64 runs follow the checker's iteration counts within one iteration and agree to
1e-8; FP32 runs reach hypergradients within 1e-4 relative error of the checker's
high-accuracy reference (the stated bar for hypergradients)."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import synth
from oracle import recycle as orc
from oracle.krylov import rcg
from tests.gpu_util import DEV, make, packed, r32, rel, split

pytestmark = pytest.mark.gpu


def lower_points(prob, th, gtol=1e-8):
    xs, _ = prob.solve_lower(th, gtol=gtol)
    return xs


def small_wl(sizes=((48, 52), (33, 70)), N=3, f=5, rb=2, seed=1):
    return synth.uneven_foe(list(sizes), n_filters=N, f=f, blur_radius=rb, seed=seed)


@pytest.mark.parametrize("precision, sizes", [("fp64", ((48, 52), (33, 70))), ("fp32", ((48, 52), (33, 70))),
                                              ("fp32", ((48, 52), (33, 72)))], ids=["fp64", "fp32", "fp32-tma"])
def test_plain_cg_matches_checker(precision, sizes):
    """fp32-tma: every width a multiple of 4, so the Hessian action runs the TMA-staged kernel and the
    Krylov dot products come from the separate chunk pass."""
    wl = small_wl(sizes=sizes)
    P, prob, dt = make(wl, precision, max_recycle=4, max_basis=60)
    assert P.hvp_tma() == (precision == "fp32" and all(w % 4 == 0 for _, w in sizes))
    th = r32(wl.theta0) if precision == "fp32" else wl.theta0
    xs = [r32(x) for x in lower_points(prob, th)] if precision == "fp32" else lower_points(prob, th)
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w = P.zeros()
    tol = 1e-8 if precision == "fp64" else 1e-6
    info = P.hessian_solve(w, recycle=False, tol=tol, relative=True, maxit=3000)
    ws = split(w, P.sizes)
    hg = P.hypergrad(w, per_pair=True)[1].cpu().numpy()
    for k in range(P.K):
        g = prob.rhs(k, xs[k])
        out = rcg(prob.apply_H(k, xs[k], th), g, np.zeros_like(g), None, None, tol=tol * np.linalg.norm(g),
                  maxit=3000)
        wref = prob.reference_w(k, xs[k], th)
        hg_ref = prob.Jw(k, xs[k], th, wref)
        if precision == "fp64":
            assert abs(info[k]["iters"] - out["iters"]) <= 1, (info[k]["iters"], out["iters"])
            assert rel(ws[k], out["w"]) < 1e-8
        assert rel(hg[k], hg_ref) < 1e-4, rel(hg[k], hg_ref)


def test_recycled_sequence_fp64_matches_checker():
    """Three systems along a theta path, RGen-L(R) refresh between them: the GPU's recycled CG
    takes the checker's iteration counts (+-1) and reaches the same hypergradients."""
    wl = small_wl(sizes=((40, 44),), N=3, seed=4)
    P, prob, dt = make(wl, "fp64", max_recycle=6, max_basis=60)
    th = wl.theta0.copy()
    rng = np.random.default_rng(0)
    U = C = Z = None
    V = None
    w_prev = None
    s = 6
    for i in range(3):
        xs = lower_points(prob, th, gtol=1e-8)
        x = xs[0]
        theta = torch.tensor(th, dtype=torch.float64, device=DEV)
        P.set_point(theta, packed(xs, dt))
        AH = prob.apply_H(0, x, th)
        if V is not None:
            P.ritz_update("RGen-L(R)", s)
            Up = U if U is not None else np.zeros((x.size, 0))
            U, C, Z, mu = orc.refresh(Up, V, AH, lambda v: prob.Jw(0, x, th, v.reshape(x.shape)), s, "rgsv", "L", "R")
            assert P.recycle_dim(0) == U.shape[1]
            # nearly the same recycle space: the Ritz-GSV selection passes through T^{-1}, so its
            # principal angles follow the rounding of the chosen basis of range(W) (an SVD here, a
            # pivoted Cholesky factor on the GPU): cosines of 0.9986-0.99995 on this sequence
            blob = P.recycle_export(0)
            n = x.size
            Ug = np.frombuffer(blob[32:32 + s * n * 8], dtype=np.float64).reshape(s, n).T
            Qa, _ = np.linalg.qr(Ug)
            Qb, _ = np.linalg.qr(U)
            cosines = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
            assert cosines.min() > 0.95 and cosines.mean() > 0.99, (i, cosines)
        g = prob.rhs(0, x)
        w0 = np.zeros_like(g) if w_prev is None else w_prev
        out = rcg(AH, g, w0, U, C, tol=1e-7 * np.linalg.norm(g), maxit=2000, kmax_store=60)
        wg = packed([w0.reshape(x.shape)], dt)
        info = P.hessian_solve(wg, recycle=True, tol=1e-7, relative=True, warm_start=True, maxit=2000)
        assert abs(info[0]["iters"] - out["iters"]) <= 1, (i, info[0]["iters"], out["iters"])
        assert rel(wg.cpu().numpy(), out["w"]) < 1e-7
        V = out["V"]
        w_prev = out["w"]
        th = th - 0.05 * rng.standard_normal(th.shape) * 0.1


@pytest.mark.parametrize("sizes", [((64, 64), (40, 90)), ((37, 45), (100, 123)), ((64, 64), (41, 92))],
                         ids=["aligned", "ragged", "tma"])
def test_refresh_invariants_fp32(sizes):
    """After bl_ritz_update: C = H U and C^T C = I on the exported recycle space (Section 2.2.2).
    "aligned": every image a multiple of 4 pixels (16-byte staging of the tall-skinny kernels);
    "ragged": odd sizes and an image spanning several 4096-pixel chunks with a short tail;
    "tma": every width a multiple of 4, so the refresh's multi-column Hessian actions (on W~ and U)
    run the TMA-staged kernel."""
    wl = small_wl(sizes=sizes, N=4, seed=7)
    P, prob, dt = make(wl, "fp32", max_recycle=8, max_basis=60)
    assert P.hvp_tma() == all(w % 4 == 0 for _, w in sizes)
    th = r32(wl.theta0)
    xs = [r32(x) for x in lower_points(prob, th, gtol=1e-8)]
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    P.set_point(theta, packed(xs, dt))
    w = P.zeros()
    P.hessian_solve(w, recycle=True, tol=1e-5, store_basis=True)
    for kind, variant in [("Ritz-S", "outer"), ("RGen-L(R)", "outer"), ("HRitz-L", "outer"), ("Ritz-S", "inner")]:
        P.set_point(theta, packed(xs, dt))
        w2 = P.zeros()
        P.hessian_solve(w2, recycle=False, tol=1e-5, store_basis="lanczos" if variant == "inner" else True)
        P.ritz_update(kind, 8, variant=variant)
        for k in range(P.K):
            s = P.recycle_dim(k)
            assert s == 8
            blob = P.recycle_export(k)
            h, wd = P.sizes[k]
            n = h * wd
            arr = np.frombuffer(blob[32:32 + 3 * s * n * 4], dtype=np.float32).astype(np.float64)
            U = arr[:s * n].reshape(s, n).T
            Cm = arr[s * n:2 * s * n].reshape(s, n).T
            np.testing.assert_allclose(Cm.T @ Cm, np.eye(s), atol=2e-4)
            HU = np.stack([prob.lowers[k].hvp(xs[k], th, U[:, j].reshape(h, wd)).ravel() for j in range(s)], 1)
            assert np.linalg.norm(HU - Cm) / np.linalg.norm(Cm) < 1e-3, kind


def test_lower_solve_first_order_condition():
    wl = small_wl(sizes=((50, 60), (23, 31)), N=3, seed=9)
    for precision, gtol in [("fp64", 1e-9), ("fp32", 1e-5)]:
        P, prob, dt = make(wl, precision)
        th = r32(wl.theta0) if precision == "fp32" else wl.theta0
        theta = torch.tensor(th, dtype=torch.float64, device=DEV)
        x = P.zeros()
        info = P.lower_solve(theta, x, gtol=gtol, relative=True, max_iters=4000)
        xs = split(x, P.sizes)
        for k, ll in enumerate(prob.lowers):
            g0 = np.linalg.norm(ll.grad(np.zeros_like(xs[k]), th))
            gn = np.linalg.norm(ll.grad(xs[k], th))
            assert gn <= 3 * gtol * g0, (precision, k, gn / g0, info[k])
            assert info[k]["status"] == 0


def test_lower_solve_trajectory_fp64_matches_checker():
    """A fixed number of L-BFGS iterations (history 4, so the (s, y) ring wraps several times)
    from x = 0: the GPU's compact-form direction, Armijo backtracking and history updates follow
    the checker's two-loop L-BFGS iterate for iterate."""
    from oracle.lbfgs import lbfgs
    wl = small_wl(sizes=((37, 45), (20, 26)), N=3, seed=21)
    P, prob, dt = make(wl, "fp64")
    th = wl.theta0
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    for iters in (3, 40):
        x = P.zeros()
        info = P.lower_solve(theta, x, gtol=0.0, relative=False, max_iters=iters, history=4, max_backtrack=30,
                             armijo_slack=0.0, allow_noconv=True)
        xs = split(x, P.sizes)
        for k, ll in enumerate(prob.lowers):
            h, w = xs[k].shape
            xr, out = lbfgs(lambda z: ll.value(z.reshape(h, w), th), lambda z: ll.grad(z.reshape(h, w), th).ravel(),
                            np.zeros(h * w), gtol=0.0, m=4, maxit=iters, max_backtrack=30)
            assert info[k]["iters"] == out["iters"] == iters
            assert rel(xs[k], xr) < 1e-9, (iters, k, rel(xs[k], xr))
            assert abs(info[k]["value"] - out["f"]) <= 1e-10 * abs(out["f"])


def test_lower_solve_graph_matches_stream():
    """The L-BFGS loop launched as one CUDA graph gives the host-polled loop's iterations and
    bit-identical iterates (the host-polled loop runs while profiling is enabled)."""
    wl = small_wl(sizes=((64, 70), (33, 40), (90, 31)), N=3, seed=23)
    P, prob, dt = make(wl, "fp32")
    theta = torch.tensor(r32(wl.theta0), dtype=torch.float64, device=DEV)
    outs = []
    for prof in (True, False, False):
        P.profile(prof)
        x = P.zeros()
        info = P.lower_solve(theta, x, gtol=1e-5, relative=True, max_iters=500, history=6)
        outs.append(([d["iters"] for d in info], [d["value"] for d in info], x.cpu().numpy()))
    P.profile(False)
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert outs[0][1] == outs[1][1] == outs[2][1]
    assert np.array_equal(outs[0][2], outs[1][2]) and np.array_equal(outs[1][2], outs[2][2])


def test_full_hypergradient_fp32():
    """Lower solve, Hessian solve and J w on the GPU (FP32) against the checker's reference."""
    wl = small_wl(sizes=((56, 56), (40, 72)), N=4, seed=11)
    P, prob, dt = make(wl, "fp32", max_recycle=8, max_basis=60)
    th = r32(wl.theta0)
    theta = torch.tensor(th, dtype=torch.float64, device=DEV)
    x = P.zeros()
    P.lower_solve(theta, x, gtol=1e-6)
    xs = split(x, P.sizes)
    w = P.zeros()
    P.hessian_solve(w, recycle=False, tol=1e-6)
    mean = P.hypergrad(w).cpu().numpy()
    refs = [prob.Jw(k, xs[k], th, prob.reference_w(k, xs[k], th)) for k in range(P.K)]
    assert rel(mean, np.mean(refs, axis=0)) < 1e-4


def test_status_codes():
    wl = small_wl(sizes=((20, 20),), N=2, seed=2)
    P, prob, dt = make(wl, "fp32", max_recycle=4, max_basis=10)
    from paper_2412_08264_gb300 import _lib as L
    w = P.zeros()
    with pytest.raises(L.BLError) as e:
        P.hessian_solve(w)                       # no point set yet
    assert e.value.status == L.BL_ESTATE
    theta = torch.tensor(r32(wl.theta0), dtype=torch.float64, device=DEV)
    P.set_point(theta, P.zeros())
    info = P.hessian_solve(w, recycle=False, tol=1e-12, maxit=1, allow_noconv=True)
    assert info[0]["status"] == L.BL_ENOCONV and info[0]["iters"] == 1
    with pytest.raises(L.BLError) as e:
        P.ritz_update("Ritz-S", 5)               # s above max_recycle
    assert e.value.status == L.BL_EINVAL
    with pytest.raises(L.BLError) as e:
        P.recycle_import(0, b"\x00" * 16)        # truncated checkpoint
    assert e.value.status == L.BL_EINVAL
    bad = torch.full((400,), float("nan"), dtype=torch.float32, device=DEV)
    with pytest.raises(L.BLError) as e:
        P.hessian_solve(P.zeros(), g=bad, recycle=False, warm_start=False)   # non-finite right-hand side
    assert e.value.status == L.BL_EBREAKDOWN


def test_graph_loop_matches_stream_loop():
    """The recycled-CG loop launched as one CUDA graph (WHILE node, device-side condition) gives the
    same iterations and bit-identical solutions as the host-polled stream loop."""
    wl = small_wl(sizes=((64, 70), (33, 40), (90, 31)), N=3, seed=17)
    P, prob, dt = make(wl, "fp32", max_recycle=6, max_basis=40)
    th = r32(wl.theta0)
    xs = [r32(x + 0.01) for x in wl.x_star]
    P.set_point(torch.tensor(th, dtype=torch.float64, device=DEV), packed(xs, dt))
    w0 = P.zeros()
    P.hessian_solve(w0, recycle=False, tol=1e-4, store_basis=True, graph=False)
    P.ritz_update("RGen-L(R)", 6)
    outs = []
    for graph in (False, True, True):
        w = P.zeros()
        info = P.hessian_solve(w, recycle=True, tol=1e-6, store_basis=False, graph=graph)
        assert P.graph_used() == graph
        outs.append(([i["iters"] for i in info], w.cpu().numpy()))
    for iters, w in outs[1:]:
        assert iters == outs[0][0]
        assert np.array_equal(w, outs[0][1])

