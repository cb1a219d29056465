"""Pins for the lower-level solver and the full hypergradient (Section 2.1, Section 5).

Finite differences of the upper-level loss through the lower-level solve fix
the sign and size of the hypergradient; the dense Cholesky reference fixes
the reference solve; L-BFGS is pinned by the first-order condition and the
Tikhonov closed form (test_oracle_functional).
"""
import numpy as np
import pytest

from paper_2412_08264_gb300 import synth
from oracle.bilevel import BilevelProblem, gradient_descent, Adam
from oracle.krylov import cg


def tiny_foe(seed=0, h=9, w=10):
    wl = synth.small_foe(h, w, n_filters=2, f=3, blur_radius=2, seed=seed)
    # make the lower level well conditioned enough for tight FD
    wl.theta0[0::10] = -1.0
    return wl


def test_lbfgs_reaches_first_order_condition():
    wl = tiny_foe()
    prob = BilevelProblem(wl)
    xs, infos = prob.solve_lower(wl.theta0, gtol=1e-10)
    g = prob.lowers[0].grad(xs[0], wl.theta0)
    assert np.linalg.norm(g) <= 1e-10
    assert infos[0]["f"] < prob.lowers[0].value(np.zeros_like(xs[0]), wl.theta0)


def test_reference_w_dense_equals_cg():
    wl = tiny_foe(1)
    prob = BilevelProblem(wl)
    xs, _ = prob.solve_lower(wl.theta0, gtol=1e-10)
    wd = prob.reference_w(0, xs[0], wl.theta0)
    H = prob.apply_H(0, xs[0], wl.theta0)
    g = prob.rhs(0, xs[0])
    wc, _, _ = cg(H, g, np.zeros_like(g), 1e-14 * np.linalg.norm(g), 10000)
    np.testing.assert_allclose(wd, wc, rtol=1e-8, atol=1e-10 * np.abs(wd).max())


def newton_lower(prob, theta, x0s, tol=1e-13, maxit=60):
    """Lower-level solves by damped Newton on the dense Hessian (tiny images only)."""
    out = []
    for k, ll in enumerate(prob.lowers):
        x = x0s[k].copy()
        for _ in range(maxit):
            g = ll.grad(x, theta).reshape(-1)
            if np.linalg.norm(g) < tol:
                break
            d = -np.linalg.solve(ll.dense_hessian(x, theta), g).reshape(x.shape)
            t, f0 = 1.0, ll.value(x, theta)
            while ll.value(x + t * d, theta) > f0 + 1e-4 * t * float(g @ d.reshape(-1)) and t > 1e-8:
                t *= 0.5
            x = x + t * d
        out.append(x)
    return out


@pytest.mark.parametrize("reg", ["foe", "tv"])
def test_hypergradient_matches_fd_of_upper_loss(reg, rng):
    """Central differences of L(theta) through exact lower solves against (1/K) sum_k J_k w_k."""
    if reg == "foe":
        wl = tiny_foe(2)
        wl.pairs = wl.pairs * 2
        wl.x_star = wl.x_star + [np.roll(wl.x_star[0], 2, axis=1)]
        wl.noise = wl.noise + [np.roll(wl.noise[0], 3, axis=0)]
    else:
        wl = synth.tv_32()
        wl.pairs = [synth.PairSpec(10, 11, 1.5, 2, 0.01)]
        wl.x_star = [wl.x_star[0][:10, :11]]
        wl.noise = [wl.noise[0][:10, :11]]
        wl.theta0 = np.array([-2.0])
    prob = BilevelProblem(wl)
    th = wl.theta0
    xs, _ = prob.solve_lower(th, gtol=1e-6)
    xs = newton_lower(prob, th, xs)
    ws = [prob.reference_w(k, xs[k], th) for k in range(prob.K)]
    hg = prob.hypergradient(th, xs, ws)
    h = 1e-5
    for _ in range(3):
        d = rng.standard_normal(prob.p)
        d = d / np.linalg.norm(d)
        fd = (prob.loss(newton_lower(prob, th + h * d, xs)) -
              prob.loss(newton_lower(prob, th - h * d, xs))) / (2 * h)
        an = float(hg @ d)
        assert abs(fd - an) < 1e-6 * max(abs(an), 1e-2 * np.linalg.norm(hg)), (fd, an)


def test_gradient_descent_decreases_upper_loss():
    """Algorithms 1-2 on the 32x32 TV workload (three steps): the Armijo test guarantees descent."""
    wl = synth.tv_32()
    prob = BilevelProblem(wl)
    log = []

    def solve(k, xh, th, g):
        return prob.reference_w(k, xh, th)

    theta, xhats, thetas = gradient_descent(prob, wl.theta0, 3, solve, gtol_lower=1e-8, log=log)
    losses = [e["loss"] for e in log]
    xs0, _ = prob.solve_lower(wl.theta0, gtol=1e-8)
    assert losses[0] < prob.loss(xs0)
    assert all(b < a for a, b in zip(losses, losses[1:]))


def test_adam_closed_form_first_step():
    """First Adam step moves every coordinate by lr * sign(g) (bias correction, eps -> 0)."""
    opt = Adam(lr=1e-2, eps=0.0)
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.1, 2e-3])
    np.testing.assert_allclose(opt.step(th, g), th - 1e-2 * np.sign(g), rtol=1e-12)


class _ScalarBilevel:
    """A one-parameter bilevel problem with closed forms, for listing Algorithm 1 by hand.

    Lower level Phi(x, theta) = 1/2 (x - theta)^2, so x^(theta) = theta, H = 1 and
    D^2_{theta x} Phi = -1; upper loss L = 1/2 a (x^ - c)^2.  Then grad ell = a (x^ - c),
    w = grad ell and the hypergradient (eq. (2.7)) is -(-1) w = a (theta - c).  Every lower
    solve is recorded, so the test sees each Armijo trial point."""

    K = 1

    def __init__(self, a, c):
        self.a, self.c = a, c
        self.trials = []

    def solve_lower(self, theta, x0s=None, gtol=1e-8):
        th = float(np.asarray(theta).ravel()[0])
        self.trials.append(th)
        return [np.array([th])], [{}]

    def loss(self, xhats):
        return 0.5 * self.a * float((xhats[0][0] - self.c) ** 2)

    def rhs(self, k, xhat):
        return self.a * (xhat - self.c)

    def hypergradient(self, theta, xhats, ws):
        return np.mean([w for w in ws], axis=0)


def _identity_solve(k, xhat, theta, g):
    return np.array(g, dtype=np.float64)


@pytest.mark.parametrize("eta, trials, steps, accepted", [
    # L = 0.75 theta^2, theta0 = 1, beta0 = 1, rho = 1/2, eta = 1e-4:
    #   step 1: d = 1.5;  trial beta rho^0 = 1 -> theta = -0.5, L = 0.1875 < 0.75 - 2.25e-4: accept; beta = 2
    #   step 2: d = -0.75; trial 2 -> theta = 1.0 (L = 0.75, reject); trial 1 -> theta = 0.25 (accept); beta = 2
    #   step 3: d = 0.375; trial 2 -> theta = -0.5 (reject); trial 1 -> theta = -0.125 (accept)
    (1e-4, [1.0, -0.5, 1.0, 0.25, -0.5, -0.125], [1.0, 1.0, 1.0], [1.0, -0.5, 0.25, -0.125]),
    # the same problem with eta = 0.6, where the sufficient-decrease term decides:
    #   step 1: trial 1 -> -0.5: 0.1875 < 0.75 - 0.6 * 2.25 fails; trial 0.5 -> 0.25: 0.046875 < 0.075: accept; beta = 1
    #   step 2: d = 0.375; trial 1 -> -0.125: 0.01172 < -0.0375 fails; trial 0.5 -> 0.0625: 0.00293 < 0.00469: accept
    #   step 3: d = 0.09375; trial 1 -> -0.03125 fails; trial 0.5 -> 0.015625: 1.83e-4 < 2.93e-4: accept
    (0.6, [1.0, -0.5, 0.25, -0.125, 0.0625, -0.03125, 0.015625], [0.5, 0.5, 0.5], [1.0, 0.25, 0.0625, 0.015625]),
])
def test_gradient_descent_lists_every_armijo_trial(eta, trials, steps, accepted):
    """Algorithms 1-2 on a worked case: the trial points beta rho^{j-1}, the sufficient-decrease test
    L(theta_j) < L(theta) - eta beta rho^{j-1} ||d||^2 and the next initial step 2 beta rho^{j-1} are
    fixed by the listing above (a dropped doubling, rho^j for rho^{j-1}, a flipped step sign or
    ||d|| for ||d||^2 each change the list)."""
    prob = _ScalarBilevel(a=1.5, c=0.0)
    log = []
    theta, xhats, thetas = gradient_descent(prob, np.array([1.0]), 3, _identity_solve, beta0=1.0, rho=0.5,
                                            eta=eta, log=log)
    np.testing.assert_allclose(prob.trials, trials, rtol=0, atol=1e-15)
    np.testing.assert_allclose([e["step_len"] for e in log], steps, rtol=0, atol=0)
    np.testing.assert_allclose([float(t[0]) for t in thetas], accepted, rtol=0, atol=1e-15)
    np.testing.assert_allclose([e["loss"] for e in log], [0.75 * t ** 2 for t in accepted[1:]], rtol=1e-15)
    assert float(theta[0]) == accepted[-1] and float(xhats[0][0]) == accepted[-1]
