"""The differentiation pattern at the size of the 8 x 1024^2 workload (24 7x7 filters, p = 1200).

The lower-level solve plus adjoint runs as the torch.autograd.Function LowerLevelSolve (forward:
L-BFGS lower solve; backward: recycled Hessian solve and J w, eqs. (2.4)-(2.7)).

  - FD: on a reduced pair set with the same filter shape (24 7x7 filters), the backward pass against
    the FP64 checker's hypergradient and against central finite differences of the upper loss along
    20 random directions (h = 1e-3).
  - Checkpointing: 30 Adam steps (Section 5.2, step 1e-2) at full size through the autograd
    Function, once straight through and once resumed at step 15 from a checkpoint (the engine's
    state: recycle spaces with their stored bases, x^, w, plus Adam's moments) in a fresh problem;
    the two end at bit-identical theta."""
import numpy as np
import pytest
import torch

from paper_2412_08264_gb300 import api, synth
from paper_2412_08264_gb300.autograd import lower_level_solve
from paper_2412_08264_gb300.outer import Engine
from tests.gpu_util import DEV, make, packed, rel

pytestmark = pytest.mark.gpu


def test_config4_filters_backward_matches_checker_and_fd():
    # small images keep the FP64 stencils (1/64 of the FP32 rate on this part) cheap: every lower
    # solve of the 40 finite differences runs L-BFGS with 24 7x7 filters in FP64
    wl = synth.uneven_foe([(12, 16), (10, 20)], n_filters=24, f=7, blur_radius=2, seed=44)
    for j in range(24):
        wl.theta0[j * 50] = -1.5          # stronger regularisation: well-conditioned lower solves
    P, prob, dt = make(wl, "fp64", max_recycle=8, max_basis=40)
    assert P.p == 1200
    # the forward solve at theta to a relative gradient of 1e-9 (compared with the checker below)
    eng = Engine(P, strategy="Ritz-S", s=8, rtol=1e-12, lower_gtol=1e-9, lower_max_iters=3000, maxit=8000,
                 refresh="inner")
    xstar = packed(prob.x_star, dt)
    theta = torch.tensor(wl.theta0, dtype=torch.float64, device=DEV, requires_grad=True)

    def loss_of(th):
        x = lower_level_solve(th, eng)
        return 0.5 * ((x - xstar) ** 2).sum() / P.K

    L = loss_of(theta)
    L.backward()
    grad = theta.grad.cpu().numpy()
    xs, _ = prob.solve_lower(wl.theta0, gtol=5e-9)
    ws = [prob.reference_w(k, xs[k], wl.theta0) for k in range(P.K)]
    ref = prob.hypergradient(wl.theta0, xs, ws)
    assert rel(grad, ref) < 1e-6, rel(grad, ref)
    # central differences at h = 1e-3: O(h^2) truncation of the loss's third derivative and the lower
    # solves' stopping error / 2h; held to 1e-3 of max(|g . d|, 1e-2 ||g||).  The 40 lower solves stop
    # at a relative gradient of 1e-7: near 1e-9 the FP64 Armijo test stops resolving decreases of Phi
    # and every step spends its 30 halvings (FP64 stencils run at 1/64 of the FP32 rate on this part),
    # while 1e-7 already keeps the difference noise ~1e-5 of the bar's scale
    eng.lower_gtol = 1e-7
    eng.lower_max_iters = 1500
    rng = np.random.default_rng(4)
    h = 1e-3
    for _ in range(20):
        d = rng.standard_normal(P.p)
        d /= np.linalg.norm(d)
        dd = torch.tensor(d, dtype=torch.float64, device=DEV)
        with torch.no_grad():
            lp = float(loss_of(theta.detach() + h * dd))
            lm = float(loss_of(theta.detach() - h * dd))
        fd = (lp - lm) / (2 * h)
        an = float(grad @ d)
        assert abs(fd - an) < 1e-3 * max(abs(an), 1e-2 * np.linalg.norm(grad)), (fd, an)


def _problem(wl, y, xs):
    return api.from_workload(wl, y, xs, max_recycle=8, max_basis=24)


def _adam(eng, xstar, theta, m, v, t0, t1, K):
    for t in range(t0 + 1, t1 + 1):
        th = torch.tensor(theta, dtype=torch.float64, device=DEV, requires_grad=True)
        x = lower_level_solve(th, eng)
        L = 0.5 * ((x - xstar) ** 2).sum() / K
        L.backward()
        g = th.grad.cpu().numpy()
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        theta = theta - 1e-2 * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    return theta, m, v


def test_config4_adam_checkpoint_resume_is_bit_identical():
    wl = synth.batch_1024()
    assert len(wl.pairs) == 8 and wl.pairs[0].height == 1024 and wl.n_params == 1200
    xs = torch.tensor(np.concatenate([x.ravel() for x in wl.x_star]), dtype=torch.float32, device=DEV)
    nz = torch.tensor(np.concatenate([x.ravel() for x in wl.noise]), dtype=torch.float32, device=DEV)
    P0 = api.from_workload(wl, xs, xs)
    y = P0.forward(xs) + nz
    del P0
    K = len(wl.pairs)
    kw = dict(strategy="Ritz-S", s=8, rtol=1e-4, lower_gtol=1e-5, lower_max_iters=2000, maxit=3000,
              refresh="inner")
    th0 = wl.theta0.copy()
    z = np.zeros_like(th0)
    # straight through
    PA = _problem(wl, y, xs)
    ea = Engine(PA, **kw)
    thA, _, _ = _adam(ea, xs, th0, z, z, 0, 30, K)
    del ea, PA
    # 15 steps, checkpoint, fresh problem, 15 more
    PB = _problem(wl, y, xs)
    eb = Engine(PB, **kw)
    th15, m15, v15 = _adam(eb, xs, th0, z, z, 0, 15, K)
    sd = eb.state_dict()
    assert any(PB.basis_size(k) > 0 for k in range(K)) and PB.recycle_dim(0) == 8
    del eb, PB
    PC = _problem(wl, y, xs)
    ec = Engine(PC, **kw)
    ec.load_state_dict(sd)
    thC, _, _ = _adam(ec, xs, th15, m15.copy(), v15.copy(), 15, 30, K)
    assert np.all(np.isfinite(thA))
    assert np.array_equal(thA, thC), float(np.abs(thA - thC).max())
